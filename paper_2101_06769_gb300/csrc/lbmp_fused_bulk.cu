// lbmp_fused_bulk.cu -- the fused D3Q27 FP32 step with its g staging done by
// the bulk-copy (TMA) engine.
//
// Same work decomposition and per-cell arithmetic as lbmp_fused.cu; the
// difference is how the pulled g of a plane reaches shared memory.  Instead
// of one 4-byte cp.async per population and cell (tile and ring), each CTA
// copies, for every direction a and every output row y of the tile plus its
// ring (TY + 2 rows), the (TX+8)-float window [x0-4, x0+TX+4) of the source
// row y - c_y of plane z - c_z: a 16-byte aligned run that contains the
// pulled value of every tile and ring cell of that row (x - c_x lies in
// [x0-2, x0+TX+1]).  27 x (TY+2) bulk copies per plane (a row
// that wraps around the periodic x boundary is split, nx being a multiple of
// 4), completed on an mbarrier with a transaction count; the threads then
// read the window at column x - x0 + 4 - c_x.  At a wall plane a bounced
// direction stages the opposite population of the row itself (column
// x - x0 + 4).  Every wait on the mbarrier is bounded in time (the handle's
// wait limit, %globaltimer); when a wait runs out the kernel records it in
// the handle's status word and returns (a wait runs out only when an
// expected copy never lands, so no copy of that CTA is left in flight).
//
// Requires nx % 4 == 0 (16-byte aligned rows); other grids use the
// cp.async kernel.
#include "lbmp_internal.h"
#include "lbmp_tile.cuh"

namespace lbmp {

namespace {

using namespace tile;

constexpr int WX = TX + 8;        // window width (floats): [x0-4, x0+TX+4)
constexpr int WR = TY + 2;        // window rows: tile rows and the two ring rows
constexpr int WIN = Q3 * WR * WX;  // floats of one staged plane
constexpr unsigned kPlaneBytes = sizeof(float) * WIN;

struct DirPtrs {
    const float* fin[Q3];
    const float* gin[Q3];
    float* fout[Q3];
    float* gout[Q3];
};

struct BulkArgs {
    int tiles_x, tiles_y, chunk, nitems;
};

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}
// wait for the phase of the given parity, at most limit_ns; false when it ran out
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned long long limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}
__device__ __forceinline__ void bulk_copy(float* dst, const float* src, unsigned bytes, unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Issue the copies of plane zz (phi ghost planes map to the wall plane) into
// the window buffer win; thread 0 arms the barrier with the plane's bytes.
__device__ __forceinline__ void issue_plane(const DevParams& p, const DirPtrs& D, int tid, int x0, int y0, int zz,
                                            float* win, unsigned long long* bar)
{
    const int pz = plane_src(p, zz);
    const bool lo = !p.vert_periodic && pz == 0, hi = !p.vert_periodic && pz == p.nz - 1;
    const int nxy = p.nx * p.ny;
    if (tid == 0) mbar_expect(bar, kPlaneBytes + p.test_extra_tx);
    fence_proxy_async();
    for (int k = tid; k < Q3 * WR; k += NT) {
        const int a = k / WR, r = k % WR;
        const int cx = Lat<3>::cx(a), cy = Lat<3>::cy(a), cz = Lat<3>::cz(a);
        (void)cx;
        const bool bounced = (cz == 1 && lo) || (cz == -1 && hi);
        const int dir = bounced ? Lat<3>::opp(a) : a;
        int zs = bounced ? pz : pz - cz;
        zs = zs < 0 ? zs + p.nz : (zs >= p.nz ? zs - p.nz : zs);
        const int ys = pmod(y0 - 1 + r - (bounced ? 0 : cy), p.ny);
        const float* row = D.gin[dir] + (zs * nxy + ys * p.nx);
        float* dst = win + (a * WR + r) * WX;
        int x = pmod(x0 - 4, p.nx), left = WX;
        while (left > 0) {
            const int len = min(left, p.nx - x);
            bulk_copy(dst, row + x, (unsigned)(len * sizeof(float)), bar);
            dst += len;
            left -= len;
            x = 0;
        }
    }
}

// pulled g of direction a for the cell at window column c (= x - x0 + 4) of
// window row r, from a staged plane with wall flags lo / hi
template <bool Walls>
__device__ __forceinline__ float win_at(const float* win, int a, int r, int c, bool lo, bool hi)
{
    const int cx = Lat<3>::cx(a), cz = Lat<3>::cz(a);
    const bool bounced = Walls && ((cz == 1 && lo) || (cz == -1 && hi));
    return win[(a * WR + r) * WX + c - (bounced ? 0 : cx)];
}

template <bool Walls>
struct GFromWin {
    const float* win;
    int r, c;
    bool lo, hi;
    __device__ __forceinline__ float operator()(int a) const { return win_at<Walls>(win, a, r, c, lo, hi); }
};

template <bool Walls>
__device__ __forceinline__ void phi_of_plane(const ThreadGeo& T, const float* win, bool lo, bool hi,
                                             float2* phi_plane)
{
    float h, l;
    if (T.tid < NRING) {
        phi_sum<3>(GFromWin<Walls>{win, T.ly + 1, T.lx + 4, lo, hi}, h, l);
        phi_plane[T.rslot] = make_float2(h, l);
    }
    phi_sum<3>(GFromWin<Walls>{win, T.ty + 1, T.tx + 4, lo, hi}, h, l);
    phi_plane[T.oslot] = make_float2(h, l);
}

// wait for plane zz in win, then its phi; false when the wait ran out
__device__ __forceinline__ bool finish_plane(const DevParams& p, const ThreadGeo& T, int zz, const float* win,
                                             unsigned long long* bar, unsigned parity, float2* phi_plane)
{
    if (!mbar_wait(bar, parity, p.wait_ns)) return false;
    const int pz = plane_src(p, zz);
    const bool lo = !p.vert_periodic && pz == 0, hi = !p.vert_periodic && pz == p.nz - 1;
    if (lo || hi)
        phi_of_plane<true>(T, win, lo, hi, phi_plane);
    else
        phi_of_plane<false>(T, win, false, false, phi_plane);
    return true;
}

__device__ __forceinline__ void report_timeout(const DevParams& p)
{
    if (p.status) atomicOr(p.status, kStatusWaitTimeout);
}

// planes [z0, z1) of the tile at (x0, y0); false when a wait ran out
__device__ __forceinline__ bool bulk_segment(const DevParams& p, const DirPtrs& Dp, const ThreadGeo& T, float* smem,
                                             unsigned long long* bars, unsigned& phases, int x0, int y0, int z0,
                                             int z1)
{
    float* gW = smem;                               // [2][WIN] staged windows
    float2* phiS = (float2*)(gW + 2 * WIN);         // (hi, lo) [3][RY][RX]
    float* dS = (float*)(phiS + 3 * PLANE);         // [27][NT] dh (LBMP_FUSED_DHSMEM)
    const int tid = T.tid;
    Column own;
    set_column(own, p, pmod(x0 + T.tx, p.nx), pmod(y0 + T.ty, p.ny));
    const bool valid = (x0 + T.tx < p.nx) && (y0 + T.ty < p.ny);
    // buffer of plane k: (k - z0 + 1) & 1; phases: bit b = parity of the next completion of buffer b
    int sP = 0, sC = 1, sN = 2;
    issue_plane(p, Dp, tid, x0, y0, z0 - 1, gW, &bars[0]);
    if (!finish_plane(p, T, z0 - 1, gW, &bars[0], phases & 1u, phiS + sP * PLANE)) return false;
    phases ^= 1u;
    __syncthreads();  // buffer 0 free before plane z0 + 1 is staged into it
    issue_plane(p, Dp, tid, x0, y0, z0, gW + WIN, &bars[1]);
    if (!finish_plane(p, T, z0, gW + WIN, &bars[1], (phases >> 1) & 1u, phiS + sC * PLANE)) return false;
    phases ^= 2u;
    for (int z = z0; z < z1; ++z) {
        const int cur = (z - z0 + 1) & 1, nxt = cur ^ 1;
        // g(z+1) in flight while f'(z) is loaded (the buffer of z-1 was freed by
        // the barrier that ended the previous plane)
        issue_plane(p, Dp, tid, x0, y0, z + 1, gW + nxt * WIN, &bars[nxt]);
        Plane P;
        set_plane(P, p, z);
        float fr[Q3];
        if (P.lo || P.hi)
            Unroll<Q3>::run(PullLoad<true>{Dp.fin, own, P, fr});
        else
            Unroll<Q3>::run(PullLoad<false>{Dp.fin, own, P, fr});
        if (!finish_plane(p, T, z + 1, gW + nxt * WIN, &bars[nxt], (phases >> nxt) & 1u, phiS + sN * PLANE))
            return false;
        phases ^= 1u << nxt;
        FlowMoments m;
        flow_moments<3>(m, fr);
        __syncthreads();
        if (valid) {
            const float2* pm = phiS + sP * PLANE + T.oslot;
            const float2* pc = phiS + sC * PLANE + T.oslot;
            const float2* pn = phiS + sN * PLANE + T.oslot;
            const float2 centre = pc[0];
            float grad[3], lap;
            stencil_from<3>(
                [&](int a) {
                    const int cz = Lat<3>::cz(a);
                    return (cz < 0 ? pm : (cz == 0 ? pc : pn))[Lat<3>::cy(a) * RX + Lat<3>::cx(a)];
                },
                centre, grad, lap);
            CellState s;
            float dh[27];
            flow_collide<3>(p, centre.x, grad, lap, m, s, dh);
            const int self = P.zs[1] + own.ys[1] + own.xs[1];
            const float* wc = gW + cur * WIN;
#if LBMP_FUSED_DHSMEM
#pragma unroll
            for (int a = 0; a < Q3; ++a) dS[a * NT + tid] = dh[a];
            const DhStrided dsrc{dS + tid, NT};
#else
            const DhArray dsrc{dh};
#endif
            if (P.lo || P.hi)
                collide_outputs<3>(p, s, dsrc, m, GFromWin<true>{wc, T.ty + 1, T.tx + 4, P.lo, P.hi}, centre.x,
                                   centre.y, PtrOut{Dp.fout, self}, PtrOut{Dp.gout, self});
            else
                collide_outputs<3>(p, s, dsrc, m, GFromWin<false>{wc, T.ty + 1, T.tx + 4, false, false}, centre.x,
                                   centre.y, PtrOut{Dp.fout, self}, PtrOut{Dp.gout, self});
        }
        __syncthreads();
        const int t = sP;
        sP = sC;
        sC = sN;
        sN = t;
    }
    return true;
}

__global__ void __launch_bounds__(NT, LBMP_FUSED_MINB) step_fused3b_kernel(DevParams p, BulkArgs A, DirPtrs Dp)
{
    extern __shared__ __align__(128) float smem_b[];
    __shared__ __align__(8) unsigned long long bars[2];
    const ThreadGeo T = thread_geo();
    if (T.tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    unsigned phases = 0;
    for (int item = blockIdx.x; item < A.nitems; item += gridDim.x) {
        const int tile = item % (A.tiles_x * A.tiles_y);
        const int chunk = item / (A.tiles_x * A.tiles_y);
        const int z0 = chunk * A.chunk;
        if (!bulk_segment(p, Dp, T, smem_b, bars, phases, (tile % A.tiles_x) * TX, (tile / A.tiles_x) * TY, z0,
                          min(z0 + A.chunk, p.nz))) {
            if (T.tid == 0) report_timeout(p);
            return;
        }
    }
}

struct BulkCfg {
    int device = -1;
    int per_sm = 0, sms = 0;
};
BulkCfg g_bulk;

}  // namespace

bool bulk_supported(const lbmp_handle* h)
{
    return h->D == 3 && h->params.storage == LBMP_FP32 && (h->grid.nx % 4) == 0;
}

cudaError_t launch_step_fused_bulk(lbmp_handle* h)
{
    const size_t smem = sizeof(float) * (2 * WIN + LBMP_FUSED_DHSMEM * Q3 * NT) + sizeof(float2) * 3 * PLANE;
    if (g_bulk.device != h->device) {
        cudaError_t e =
            cudaFuncSetAttribute(step_fused3b_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_fused3b_kernel, NT, smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        if (e != cudaSuccess) return e;
        g_bulk.per_sm = per_sm > 0 ? per_sm : 1;
        g_bulk.sms = sms;
        g_bulk.device = h->device;
    }
    DirPtrs D;
    const int s = h->parity, d = 1 - h->parity;
    for (int a = 0; a < Q3; ++a) {
        const size_t off = (size_t)a * (size_t)h->N;
        D.fin[a] = h->f[s] + off;
        D.gin[a] = h->g[s] + off;
        D.fout[a] = h->f[d] + off;
        D.gout[a] = h->g[d] + off;
    }
    BulkArgs A;
    A.tiles_x = (h->grid.nx + TX - 1) / TX;
    A.tiles_y = (h->grid.ny + TY - 1) / TY;
    const LaunchShape L = launch_shape(h, A.tiles_x * A.tiles_y, h->grid.nz, g_bulk.per_sm, g_bulk.sms);
    A.chunk = L.chunk;
    A.nitems = L.nitems;
    step_fused3b_kernel<<<L.grid, NT, smem, h->stream>>>(h->dp, A, D);
    return cudaGetLastError();
}

}  // namespace lbmp
