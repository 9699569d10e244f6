// lbmp_fused.cu -- fused single-pass D3Q27 step: phi, its isotropic
// differences, the cumulant flow collision, the phase-field collision and the
// streaming of both population sets in one kernel.
//
// Work decomposition: a CTA owns an xy tile of TX x TY cells (one thread per
// cell column) and marches through a chunk of z planes.  For plane z it needs
// phi on planes z-1, z, z+1 over the tile plus a one-cell ring.  phi = sum_a g_a
// of the post-streaming g, i.e. of exactly the values the step pulls, so each
// plane's phi is formed from the populations themselves while they are
// staged: the tile's own g(z+1) is copied asynchronously (cp.async) into
// shared memory, summed for phi and kept for the collision of plane z+1; the
// ring cells' g are loaded and summed by the first threads.  Because the step
// reads one population set and writes the other, the ring reads cannot race
// with the neighbouring tile's writes.  No phi field is stored and no
// separate phi pass runs; the only bytes beyond "every population read once
// and written once" are ring reads, which the neighbouring tiles fetch at
// about the same time (mostly L2 hits), and one extra plane per chunk.
//
// Addressing: the 27 per-direction array bases of the four population sets
// are kernel parameters (constant bank); a pulled value is base[a] plus a
// 32-bit cell index assembled from three per-axis neighbour offsets, so each
// load costs an add and a wide multiply-add.
//
// The per-cell arithmetic (lbmp_common.cuh) and its summation orders are the
// ones of the reference pair in lbmp_kernels.cu, so the two paths agree.
#include "lbmp_internal.h"

namespace lbmp {

namespace {

// tile shape and CTAs per SM (compile-time; the defaults are the measured best)
#ifndef LBMP_FUSED_TX
#define LBMP_FUSED_TX 32
#endif
#ifndef LBMP_FUSED_TY
#define LBMP_FUSED_TY 4
#endif
#ifndef LBMP_FUSED_MINB
#define LBMP_FUSED_MINB 3
#endif
// 1: f' of the plane is staged by cp.async into shared memory with the g
// copies (frees the registers of 27 loads in flight); 0: loaded to registers
#ifndef LBMP_FUSED_FSMEM
#define LBMP_FUSED_FSMEM 0
#endif
// 1: the 27 post-collision moment differences are parked in shared memory
// between the collision set-up and the output loop
#ifndef LBMP_FUSED_DHSMEM
#define LBMP_FUSED_DHSMEM 0
#endif
constexpr int TX = LBMP_FUSED_TX, TY = LBMP_FUSED_TY, NT = TX * TY;
constexpr int RX = TX + 2, RY = TY + 2;
constexpr int PLANE = RY * RX;
constexpr int NRING = 2 * RX + 2 * TY;
constexpr int Q3 = 27;
constexpr size_t kSmemBytes =
    sizeof(float) * ((2 + LBMP_FUSED_FSMEM + LBMP_FUSED_DHSMEM) * Q3 * NT + Q3 * NRING) + sizeof(float2) * 3 * PLANE;
static_assert(NRING <= NT, "one thread per ring cell");

struct DirPtrs {
    const float* fin[Q3];
    const float* gin[Q3];
    float* fout[Q3];
    float* gout[Q3];
};

// Work items: (tile, chunk of z planes), tile index fastest, so the CTAs
// running at any moment hold neighbouring tiles of the same z range and the
// ring reads of one tile are the own reads of another (L2 hits).  A
// contiguous split of the plane-columns per CTA, which balances better on
// paper, measured slower for that reason.
struct FusedArgs {
    int tiles_x, tiles_y, chunk, nitems;
};

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ int pmod(int v, int n)
{
    const int r = v % n;
    return r < 0 ? r + n : r;
}

// A column (x, y) and its upstream neighbours: xs[c+1] = x - c and
// ys[c+1] = (y - c) nx, wrapped periodically.
struct Column {
    int xs[3], ys[3];
};

__device__ __forceinline__ void set_column(Column& C, const DevParams& p, int x, int y)
{
    C.xs[0] = x + 1 == p.nx ? 0 : x + 1;
    C.xs[1] = x;
    C.xs[2] = x == 0 ? p.nx - 1 : x - 1;
    C.ys[0] = (y + 1 == p.ny ? 0 : y + 1) * p.nx;
    C.ys[1] = y * p.nx;
    C.ys[2] = (y == 0 ? p.ny - 1 : y - 1) * p.nx;
}

// A plane z and its upstream planes zs[c+1] = (z - c) nx ny; lo/hi flag the
// bottom/top plane of a walled domain, where the population arriving across
// the wall is the opposite population of the cell itself (half-way
// bounce-back).
struct Plane {
    int zs[3];
    bool lo, hi;
};

__device__ __forceinline__ void set_plane(Plane& P, const DevParams& p, int z)
{
    const int nxy = p.nx * p.ny;
    P.lo = !p.vert_periodic && z == 0;
    P.hi = !p.vert_periodic && z == p.nz - 1;
    P.zs[0] = (z + 1 == p.nz ? 0 : z + 1) * nxy;
    P.zs[1] = z * nxy;
    P.zs[2] = (z == 0 ? p.nz - 1 : z - 1) * nxy;
}

// pointer to the post-streaming population a of the cell (column C, plane P);
// Walls = false is the path of every plane that does not touch a wall
template <bool Walls, int a>
__device__ __forceinline__ const float* pulled(const float* const* base, const Column& C, const Plane& P)
{
    constexpr int cx = Lat<3>::cx(a), cy = Lat<3>::cy(a), cz = Lat<3>::cz(a);
    if (Walls && ((cz == 1 && P.lo) || (cz == -1 && P.hi)))
        return base[Lat<3>::opp(a)] + (P.zs[1] + C.ys[1] + C.xs[1]);
    return base[a] + (P.zs[cz + 1] + C.ys[cy + 1] + C.xs[cx + 1]);
}

// compile-time loop over the directions (keeps base[a] a constant-bank operand)
template <int N>
struct Unroll {
    template <class F>
    __device__ __forceinline__ static void run(const F& f)
    {
        Unroll<N - 1>::run(f);
        f.template step<N - 1>();
    }
};
template <>
struct Unroll<0> {
    template <class F>
    __device__ __forceinline__ static void run(const F&)
    {
    }
};

// plane whose phi stands for plane zz: periodic wrap, or the mirrored ghost
// at a wall (reading A17)
__device__ __forceinline__ int plane_src(const DevParams& p, int zz)
{
    if (zz >= 0 && zz < p.nz) return zz;
    if (p.vert_periodic) return pmod(zz, p.nz);
    return zz < 0 ? 0 : p.nz - 1;
}

template <bool Walls>
struct StageCopy {
    const DirPtrs& D;
    const Column& C;
    const Plane& P;
    float* gbuf;
    template <int a>
    __device__ __forceinline__ void step() const
    {
        cp_async4(gbuf + a * NT, pulled<Walls, a>(D.gin, C, P));
    }
};

template <bool Walls>
struct PullLoad {
    const float* const* base;
    const Column& C;
    const Plane& P;
    float* v;
    template <int a>
    __device__ __forceinline__ void step() const
    {
        v[a] = __ldg(pulled<Walls, a>(base, C, P));
    }
};

template <bool Walls>
struct FCopy {
    const DirPtrs& D;
    const Column& C;
    const Plane& P;
    float* fbuf;
    template <int a>
    __device__ __forceinline__ void step() const
    {
        cp_async4(fbuf + a * NT, pulled<Walls, a>(D.fin, C, P));
    }
};

template <bool Walls>
struct RingCopy {
    const DirPtrs& D;
    const Column& C;
    const Plane& P;
    float* rbuf;
    template <int a>
    __device__ __forceinline__ void step() const
    {
        cp_async4(rbuf + a * NRING, pulled<Walls, a>(D.gin, C, P));
    }
};

// Staging of plane zz, in two halves so that other loads can be issued while
// the copies are in flight.  issue: the tile's own g(zz) into gbuf (kept for
// the collision of plane zz) and the ring cells' g(zz) into rbuf, both by
// cp.async.  finish: wait, then phi = (hi, lo) of every tile and ring cell
// into phi_plane.  Each thread sums only the values it copied itself, so no
// barrier is needed in between.
__device__ __forceinline__ void stage_issue(const DevParams& p, const DirPtrs& D, const Column& own,
                                            const Column& ring, int tid, int zz, float* __restrict__ gbuf,
                                            float* __restrict__ rbuf)
{
    Plane P;
    set_plane(P, p, plane_src(p, zz));
    if (P.lo || P.hi) {  // uniform across the CTA
        Unroll<Q3>::run(StageCopy<true>{D, own, P, gbuf + tid});
        if (tid < NRING) Unroll<Q3>::run(RingCopy<true>{D, ring, P, rbuf + tid});
    } else {
        Unroll<Q3>::run(StageCopy<false>{D, own, P, gbuf + tid});
        if (tid < NRING) Unroll<Q3>::run(RingCopy<false>{D, ring, P, rbuf + tid});
    }
    cp_async_commit();
}

__device__ __forceinline__ void stage_finish(int tid, int oslot, int rslot, const float* __restrict__ gbuf,
                                             const float* __restrict__ rbuf, float2* __restrict__ phi_plane)
{
    cp_async_wait_all();
    if (tid < NRING) {
        float hi, lo;
        phi_sum<3>([&](int a) { return rbuf[a * NRING + tid]; }, hi, lo);
        phi_plane[rslot] = make_float2(hi, lo);
    }
    float hi, lo;
    phi_sum<3>([&](int a) { return gbuf[a * NT + tid]; }, hi, lo);
    phi_plane[oslot] = make_float2(hi, lo);
}

// per-thread geometry inside a tile: own cell and (for tid < NRING) ring cell
struct ThreadGeo {
    int tid, tx, ty, oslot, lx, ly, rslot;
};

__device__ __forceinline__ ThreadGeo thread_geo()
{
    ThreadGeo T;
    T.tid = threadIdx.x;
    T.tx = T.tid % TX;
    T.ty = T.tid / TX;
    T.oslot = (T.ty + 1) * RX + (T.tx + 1);
    T.lx = T.ly = T.rslot = 0;
    if (T.tid < NRING) {
        const int r = T.tid;
        if (r < RX) {
            T.lx = r - 1;
            T.ly = -1;
        } else if (r < 2 * RX) {
            T.lx = r - RX - 1;
            T.ly = TY;
        } else if (r < 2 * RX + TY) {
            T.lx = -1;
            T.ly = r - 2 * RX;
        } else {
            T.lx = TX;
            T.ly = r - 2 * RX - TY;
        }
        T.rslot = (T.ly + 1) * RX + (T.lx + 1);
    }
    return T;
}

// One segment of work: planes [z0, z1) of the tile at (x0, y0) of the domain
// described by (p, Dp).  smem holds the g staging buffers, the ring buffer and
// the three phi planes.  Ends with a barrier, so the caller may reuse shared
// memory afterwards.
__device__ __forceinline__ void fused_segment(const DevParams& p, const DirPtrs& Dp, const ThreadGeo& T, float* smem,
                                              int x0, int y0, int z0, int z1)
{
    float* gS = smem;                           // [2][27][NT]
    float* rS = smem + 2 * Q3 * NT;             // [27][NRING] ring cells' g of the plane being staged
    float2* phiS = (float2*)(rS + Q3 * NRING);  // (hi, lo) [3][RY][RX]
    float* fS = (float*)(phiS + 3 * PLANE);     // [27][NT] f' of the plane (LBMP_FUSED_FSMEM)
    float* dS = fS + LBMP_FUSED_FSMEM * Q3 * NT;  // [27][NT] dh (LBMP_FUSED_DHSMEM)
    const int tid = T.tid, oslot = T.oslot, rslot = T.rslot;
    Column own, ring;
    set_column(own, p, pmod(x0 + T.tx, p.nx), pmod(y0 + T.ty, p.ny));
    set_column(ring, p, pmod(x0 + T.lx, p.nx), pmod(y0 + T.ly, p.ny));
    const bool valid = (x0 + T.tx < p.nx) && (y0 + T.ty < p.ny);
    int sP = 0, sC = 1, sN = 2;
    stage_issue(p, Dp, own, ring, tid, z0 - 1, gS + Q3 * NT, rS);
    stage_finish(tid, oslot, rslot, gS + Q3 * NT, rS, phiS + sP * PLANE);
    stage_issue(p, Dp, own, ring, tid, z0, gS, rS);
    stage_finish(tid, oslot, rslot, gS, rS, phiS + sC * PLANE);
    for (int z = z0; z < z1; ++z) {
        const int cur = (z - z0) & 1;
        // g(z+1) and the ring copies in flight while f'(z) is loaded
        stage_issue(p, Dp, own, ring, tid, z + 1, gS + (cur ^ 1) * Q3 * NT, rS);
        Plane P;
        set_plane(P, p, z);
        FlowMoments m;
#if LBMP_FUSED_FSMEM
        if (P.lo || P.hi)
            Unroll<Q3>::run(FCopy<true>{Dp, own, P, fS + tid});
        else
            Unroll<Q3>::run(FCopy<false>{Dp, own, P, fS + tid});
        cp_async_commit();
        stage_finish(tid, oslot, rslot, gS + (cur ^ 1) * Q3 * NT, rS, phiS + sN * PLANE);
        {
            float fr[Q3];
#pragma unroll
            for (int a = 0; a < Q3; ++a) fr[a] = fS[a * NT + tid];
            flow_moments<3>(m, fr);
        }
#else
        float fr[Q3];
        if (P.lo || P.hi)
            Unroll<Q3>::run(PullLoad<true>{Dp.fin, own, P, fr});
        else
            Unroll<Q3>::run(PullLoad<false>{Dp.fin, own, P, fr});
        stage_finish(tid, oslot, rslot, gS + (cur ^ 1) * Q3 * NT, rS, phiS + sN * PLANE);
        flow_moments<3>(m, fr);
#endif
        __syncthreads();
        if (valid) {
            float nh[Q3], nl[Q3];
#pragma unroll
            for (int a = 0; a < Q3; ++a) {
                const int cz = Lat<3>::cz(a);
                const float2* pl = phiS + (cz < 0 ? sP : (cz == 0 ? sC : sN)) * PLANE;
                const float2 v = pl[oslot + Lat<3>::cy(a) * RX + Lat<3>::cx(a)];
                nh[a] = v.x;
                nl[a] = v.y;
            }
            float grad[3], lap;
            stencil_from_nb<3>(nh, nl, grad, lap);
            CellState s;
            float dh[27];
            flow_collide<3>(p, nh[13], grad, lap, m, s, dh);
            const int self = P.zs[1] + own.ys[1] + own.xs[1];
#if LBMP_FUSED_DHSMEM
#pragma unroll
            for (int a = 0; a < Q3; ++a) dS[a * NT + tid] = dh[a];
            collide_outputs<3>(p, s, DhStrided{dS + tid, NT}, m, GFromStrided{gS + cur * Q3 * NT + tid, NT}, nh[13],
                               nl[13], PtrOut{Dp.fout, self}, PtrOut{Dp.gout, self});
#else
            collide_outputs<3>(p, s, DhArray{dh}, m, GFromStrided{gS + cur * Q3 * NT + tid, NT}, nh[13], nl[13],
                               PtrOut{Dp.fout, self}, PtrOut{Dp.gout, self});
#endif
        }
        __syncthreads();
        const int t = sP;
        sP = sC;
        sC = sN;
        sN = t;
    }
}

__global__ void __launch_bounds__(NT, LBMP_FUSED_MINB) step_fused3_kernel(DevParams p, FusedArgs A, DirPtrs Dp)
{
    extern __shared__ float smem[];
    const ThreadGeo T = thread_geo();
    for (int item = blockIdx.x; item < A.nitems; item += gridDim.x) {
        const int tile = item % (A.tiles_x * A.tiles_y);
        const int chunk = item / (A.tiles_x * A.tiles_y);
        const int z0 = chunk * A.chunk;
        fused_segment(p, Dp, T, smem, (tile % A.tiles_x) * TX, (tile / A.tiles_x) * TY, z0,
                      min(z0 + A.chunk, p.nz));
    }
}

// Batch form: the work items of every member (same order as above within a
// member, members concatenated) are split over one persistent grid.  A CTA
// stages the parameters and the 108 direction bases of its current member in
// shared memory; members whose steps have run out are skipped.
__global__ void __launch_bounds__(NT, LBMP_FUSED_MINB) step_batch3_kernel(const BatchDomain* __restrict__ table,
                                                                          int ndom, int nitems)
{
    extern __shared__ float smem[];
    __shared__ DevParams sp;
    __shared__ DirPtrs sd;
    __shared__ int s_dom, s_tx, s_ty, s_chunk, s_begin, s_active;
    const ThreadGeo T = thread_geo();
    int cur = -1;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        __syncthreads();  // every thread has read the previous item's shared values
        if (threadIdx.x == 0) {
            int lo = 0, hi = ndom - 1;  // last member with item_begin <= item
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (table[mid].item_begin <= item)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            s_dom = lo;
        }
        __syncthreads();
        const int d = s_dom;
        if (d != cur) {
            const BatchDomain& B = table[d];
            if (threadIdx.x == 0) {
                sp = B.p;
                s_tx = B.tiles_x;
                s_ty = B.tiles_y;
                s_chunk = B.chunk;
                s_begin = B.item_begin;
                s_active = B.steps_left > 0;
            }
            const int par = B.parity;
            for (int k = threadIdx.x; k < 4 * Q3; k += blockDim.x) {
                const int set = k / Q3, a = k % Q3;
                const size_t off = (size_t)a * (size_t)B.p.N;
                if (set == 0) sd.fin[a] = B.f[par] + off;
                if (set == 1) sd.gin[a] = B.g[par] + off;
                if (set == 2) sd.fout[a] = B.f[par ^ 1] + off;
                if (set == 3) sd.gout[a] = B.g[par ^ 1] + off;
            }
            cur = d;
            __syncthreads();
        }
        if (!s_active) continue;  // uniform
        const int local = item - s_begin;
        const int tiles = s_tx * s_ty;
        const int tile = local % tiles;
        const int z0 = (local / tiles) * s_chunk;
        fused_segment(sp, sd, T, smem, (tile % s_tx) * TX, (tile / s_tx) * TY, z0, min(z0 + s_chunk, sp.nz));
    }
}

struct LaunchCfg {
    int device = -1;
    int grid_cap = 0;
};
LaunchCfg g_cfg;

}  // namespace

bool fused_supported(const lbmp_handle* h) { return h->D == 3 || h->D == 2; }

__global__ void batch_epilogue_kernel(BatchDomain* table, int ndom)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d < ndom && table[d].steps_left > 0) {
        table[d].parity ^= 1;
        table[d].steps_left -= 1;
    }
}

int batch3_tile_x() { return TX; }
int batch3_tile_y() { return TY; }

static int g_batch_dev = -1, g_batch_cap = 0;

// attributes and occupancy of the batch kernel (not capturable: call before capture)
cudaError_t prepare_batch3(int device)
{
    int& dev_cached = g_batch_dev;
    int& cap = g_batch_cap;
    if (dev_cached != device) {
        cudaError_t e = cudaFuncSetAttribute(step_batch3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_batch3_kernel, NT, kSmemBytes);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) return e;
        cap = (per_sm > 0 ? per_sm : 1) * sms;
        dev_cached = device;
    }
    return cudaSuccess;
}

cudaError_t launch_batch3(const BatchDomain* table, int ndom, int nitems, int device, cudaStream_t stream)
{
    if (g_batch_dev != device) return cudaErrorNotReady;  // prepare_batch3 first
    if (nitems <= 0) return cudaSuccess;
    const int grid = nitems < g_batch_cap ? nitems : g_batch_cap;
    step_batch3_kernel<<<grid, NT, kSmemBytes, stream>>>(table, ndom, nitems);
    return cudaGetLastError();
}

cudaError_t launch_batch_epilogue(BatchDomain* table, int ndom, cudaStream_t stream)
{
    if (ndom <= 0) return cudaSuccess;
    batch_epilogue_kernel<<<(ndom + 127) / 128, 128, 0, stream>>>(table, ndom);
    return cudaGetLastError();
}

cudaError_t launch_step_fused(lbmp_handle* h)
{
    if (h->D == 2) return launch_step_fused2(h);
    if (g_cfg.device != h->device) {
        cudaError_t e = cudaFuncSetAttribute(step_fused3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_fused3_kernel, NT, kSmemBytes);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        if (e != cudaSuccess) return e;
        g_cfg.grid_cap = (per_sm > 0 ? per_sm : 1) * sms;
        g_cfg.device = h->device;
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
    FusedArgs A;
    A.tiles_x = (h->grid.nx + TX - 1) / TX;
    A.tiles_y = (h->grid.ny + TY - 1) / TY;
    const int tiles = A.tiles_x * A.tiles_y;
    // chunk length: enough items to balance the persistent grid, at least 8 planes
    int chunk = h->grid.nz;
    while (chunk > 8 && (long long)tiles * ((h->grid.nz + chunk - 1) / chunk) < 4LL * g_cfg.grid_cap) chunk /= 2;
    A.chunk = chunk;
    A.nitems = tiles * ((h->grid.nz + chunk - 1) / chunk);
    const int grid = A.nitems < g_cfg.grid_cap ? A.nitems : g_cfg.grid_cap;
    step_fused3_kernel<<<grid, NT, kSmemBytes, h->stream>>>(h->dp, A, D);
    return cudaGetLastError();
}

}  // namespace lbmp
