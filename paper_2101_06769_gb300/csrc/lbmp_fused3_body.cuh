// lbmp_fused3_body.cuh -- the fused D3Q27 FP32 step kernel, its batch form
// and its launcher, for the tile shape of the including unit.
//
// The fused single-pass step: phi, its isotropic differences, the cumulant
// flow collision, the phase-field collision and the streaming of both
// population sets in one kernel.
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
//
// The including unit defines LBMP_FUSED3_LAUNCH (the launcher's name),
// LBMP_BATCH3_OPS (the name of its batch-kernel table) and, for a tile shape
// other than the default, LBMP_FUSED_TX / _TY and LBMP_TILE_NS;
// LBMP_FUSED3_WITH_COMMON adds the pieces shared by every tile shape.
// LBMP_PHASE_REDUCED = 1 builds the kernel for the reduced phase lattice
// (D3Q7 g with the first-order equilibrium and the correction term, Sec. 2.2;
// the stored previous phi u is read and replaced per cell).
#pragma once

#include <string.h>

#include "lbmp_internal.h"
#include "lbmp_tile.cuh"

namespace lbmp {

namespace {

using namespace LBMP_TILE_NS;


struct DirPtrs {
    const float* fin[Q3];
    const float* gin[QG];
    float* fout[Q3];
    float* gout[QG];
};

// Work items: (tile, chunk of z planes), tile index fastest, so the CTAs
// running at any moment hold neighbouring tiles of the same z range and the
// ring reads of one tile are the own reads of another (L2 hits).  A
// contiguous split of the plane-columns per CTA, which balances better on
// paper, measured slower for that reason.
struct FusedArgs {
    int tiles_x, tiles_y, chunk, nitems;
    float* phiu;  // reduced phase lattice: previous phi u, [k][cell]; else null
};

template <bool Walls>
struct StageCopy {
    const DirPtrs& D;
    const Column& C;
    const Plane& P;
    float* gbuf;
    template <int r>
    __device__ __forceinline__ void step() const
    {
        cp_async4(gbuf + r * NT, pulled_g<Walls, r>(D.gin, C, P));
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
    template <int r>
    __device__ __forceinline__ void step() const
    {
        cp_async4(rbuf + r * NRING, pulled_g<Walls, r>(D.gin, C, P));
    }
};

// Staging of plane zz, in two halves so that other loads can be issued while
// the copies are in flight.  issue: the tile's own g(zz) into gbuf (kept for
// the collision of plane zz) and the ring cells' g(zz) into rbuf, both by
// cp.async.  finish: wait, then phi = (hi, lo) of every tile and ring cell
// into phi_plane.  Each thread sums only the values it copied itself, so no
// barrier is needed in between.
// Reduced phase lattice: the own cells' stored phi u of plane zz is copied
// with them into ubuf ([3][NT]), so the collision finds it in shared memory.
// With kRingReg the ring threads instead load their cell's g(zz) to
// registers and write its phi at once, after issuing the own copies.

// ring cell's g(zz) loaded to registers and summed at once (kRingReg)
template <bool Walls>
__device__ __forceinline__ void ring_phi_direct(const DirPtrs& D, const Column& C, const Plane& P, float2* dst)
{
    float v[QG];
    Unroll<QG>::run(PullLoadG<Walls>{D.gin, C, P, v});
    float hi, lo;
    phi_sum_phase<3, PR>([&](int r) { return v[r]; }, hi, lo);
    *dst = make_float2(hi, lo);
}

__device__ __forceinline__ void stage_issue(const DevParams& p, const DirPtrs& D, const Column& own,
                                            const Column& ring, int tid, int rslot, int zz, float* __restrict__ gbuf,
                                            float* __restrict__ rbuf, const float* __restrict__ phiu,
                                            float* __restrict__ ubuf, float2* __restrict__ phi_plane)
{
    Plane P;
    set_plane(P, p, plane_src(p, zz));
    if constexpr (PR) {
        const int self = elem_index(P.zs[1] + own.ys[1] + own.xs[1]);
#pragma unroll
        for (int k = 0; k < 3; ++k) cp_async4(ubuf + k * NT + tid, phiu + k * p.N + self);
    }
    if (P.lo || P.hi) {  // uniform across the CTA
        Unroll<QG>::run(StageCopy<true>{D, own, P, gbuf + tid});
        if (!kRingReg && tid < NRING) Unroll<QG>::run(RingCopy<true>{D, ring, P, rbuf + tid});
    } else {
        Unroll<QG>::run(StageCopy<false>{D, own, P, gbuf + tid});
        if (!kRingReg && tid < NRING) Unroll<QG>::run(RingCopy<false>{D, ring, P, rbuf + tid});
    }
    cp_async_commit();
    if constexpr (kRingReg) {
        // the phi plane slot is free: the barrier ending the previous plane
        // separates this write from the last stencil reads of its old plane
        if (tid < NRING) {
            if (P.lo || P.hi)
                ring_phi_direct<true>(D, ring, P, phi_plane + rslot);
            else
                ring_phi_direct<false>(D, ring, P, phi_plane + rslot);
        }
    }
}

__device__ __forceinline__ void stage_finish(int tid, int oslot, int rslot, const float* __restrict__ gbuf,
                                             const float* __restrict__ rbuf, float2* __restrict__ phi_plane)
{
    cp_async_wait_all();
    if (!kRingReg && tid < NRING) {
        float hi, lo;
        phi_sum_phase<3, PR>([&](int r) { return rbuf[r * NRING + tid]; }, hi, lo);
        phi_plane[rslot] = make_float2(hi, lo);
    }
    float hi, lo;
    phi_sum_phase<3, PR>([&](int r) { return gbuf[r * NT + tid]; }, hi, lo);
    phi_plane[oslot] = make_float2(hi, lo);
}

// One segment of work: planes [z0, z1) of the tile at (x0, y0) of the domain
// described by (p, Dp).  smem holds the g staging buffers, the ring buffer and
// the three phi planes.  Ends with a barrier, so the caller may reuse shared
// memory afterwards.
__device__ __forceinline__ void fused_segment(const DevParams& p, const DirPtrs& Dp, const ThreadGeo& T, float* smem,
                                              int x0, int y0, int z0, int z1, float* __restrict__ phiu)
{
    float* gS = smem;                                    // [2][QG][NT]
    float* rS = smem + 2 * QG * NT;                      // [QG][NRING] ring cells' g of the plane being staged
    float2* phiS = (float2*)(rS + (kRingReg ? 0 : QG * NRING));  // (hi, lo) [3][RY][RX]
    float* fS = (float*)(phiS + 3 * PLANE);              // [27][NT] f' of the plane (LBMP_FUSED_FSMEM)
    float* dS = fS + LBMP_FUSED_FSMEM * Q3 * NT;         // [27][NT] dh (kDhSmem)
    float* uS = dS + (kDhSmem ? Q3 * NT : 0);            // [2][3][NT] previous phi u (reduced phase lattice)
    const int tid = T.tid, oslot = T.oslot, rslot = T.rslot;
    Column own, ring;
    set_column(own, p, pmod(x0 + T.tx, p.nx), pmod(y0 + T.ty, p.ny));
    set_column(ring, p, pmod(x0 + T.lx, p.nx), pmod(y0 + T.ly, p.ny));
    const bool valid = (x0 + T.tx < p.nx) && (y0 + T.ty < p.ny);
    int sP = 0, sC = 1, sN = 2;
    stage_issue(p, Dp, own, ring, tid, rslot, z0 - 1, gS + QG * NT, rS, phiu, uS + 3 * NT, phiS + sP * PLANE);
    stage_finish(tid, oslot, rslot, gS + QG * NT, rS, phiS + sP * PLANE);
    stage_issue(p, Dp, own, ring, tid, rslot, z0, gS, rS, phiu, uS, phiS + sC * PLANE);
    stage_finish(tid, oslot, rslot, gS, rS, phiS + sC * PLANE);
    for (int z = z0; z < z1; ++z) {
        const int cur = (z - z0) & 1;
        // g(z+1) and the ring copies in flight while f'(z) is loaded
        stage_issue(p, Dp, own, ring, tid, rslot, z + 1, gS + (cur ^ 1) * QG * NT, rS, phiu, uS + (cur ^ 1) * 3 * NT,
                    phiS + sN * PLANE);
        Plane P;
        set_plane(P, p, z);
        FlowMoments m;
#if LBMP_FUSED_FSMEM
        if (P.lo || P.hi)
            Unroll<Q3>::run(FCopy<true>{Dp, own, P, fS + tid});
        else
            Unroll<Q3>::run(FCopy<false>{Dp, own, P, fS + tid});
        cp_async_commit();
        stage_finish(tid, oslot, rslot, gS + (cur ^ 1) * QG * NT, rS, phiS + sN * PLANE);
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
        stage_finish(tid, oslot, rslot, gS + (cur ^ 1) * QG * NT, rS, phiS + sN * PLANE);
        flow_moments<3>(m, fr);
#endif
        __syncthreads();
        if (valid) {
            const float2* pm = phiS + sP * PLANE + oslot;
            const float2* pc = phiS + sC * PLANE + oslot;
            const float2* pn = phiS + sN * PLANE + oslot;
            const float2 centre = pc[0];
            float grad[3], lap;
            stencil_from<3>(
                [&](int a) {
                    const int cz = Lat<3>::cz(a);
                    return (cz < 0 ? pm : (cz == 0 ? pc : pn))[Lat<3>::cy(a) * RX + Lat<3>::cx(a)];
                },
                centre, grad, lap);
            CellState s;
            const cell_off self = P.zs[1] + own.ys[1] + own.xs[1];
            float* gcol = gS + cur * QG * NT + tid;  // this cell's staged pre-collision g
            if constexpr (kSplit) {
                // g first; its staged column then holds the moment differences
                float inv_rho, nu;
                flow_closure<3>(p, centre.x, grad, lap, m, s, inv_rho, nu);
                phase_outputs<3>(p, s, GFromStrided{gcol, NT}, centre.x, centre.y, CellOut{Dp.gout, self});
                float dh[27];
                flow_relax<3>(m, s, inv_rho, nu, dh);
#pragma unroll
                for (int a = 0; a < Q3; ++a) gcol[a * NT] = dh[a];
                flow_outputs<3>(s, DhStrided{gcol, NT}, m, CellOut{Dp.fout, self});
            } else {
                float dh[27];
                flow_collide<3>(p, centre.x, grad, lap, m, s, dh);
                if constexpr (kDhSmem) {
#pragma unroll
                    for (int a = 0; a < Q3; ++a) dS[a * NT + tid] = dh[a];
                    collide_outputs<3, PR>(p, s, DhStrided{dS + tid, NT}, m, GFromStrided{gcol, NT}, centre.x,
                                           centre.y, CellOut{Dp.fout, self}, CellOut{Dp.gout, self},
                                           PhiUStaged<3>{p, phiu, elem_index(self), uS + cur * 3 * NT + tid, NT});
                } else {
                    collide_outputs<3, PR>(p, s, DhArray{dh}, m, GFromStrided{gcol, NT}, centre.x, centre.y,
                                           CellOut{Dp.fout, self}, CellOut{Dp.gout, self},
                                           PhiUStaged<3>{p, phiu, elem_index(self), uS + cur * 3 * NT + tid, NT});
                }
            }
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
        const int z0 = p.zb + chunk * A.chunk;  // the updated planes [zb, ze) (all planes but a slab's ghosts)
        fused_segment(p, Dp, T, smem, (tile % A.tiles_x) * TX, (tile / A.tiles_x) * TY, z0,
                      min(z0 + A.chunk, p.ze), A.phiu);
    }
}

// Batch form: the members are kernel parameters, one member per blockIdx.y,
// so a member's parameters and direction bases are read from the constant
// bank at an index common to the whole CTA, as in the single-domain kernel (a
// persistent kernel that stages the current member's parameters and bases in
// shared memory reads them from there at every use, and measured 8 % slower).  gridDim.x covers the largest member's work items; a smaller member's
// spare CTAs return at once.  The parity of each member is fixed in the
// parameters: a captured graph holds one launch per step with the parities of
// that step.
struct GridMember {
    DevParams p;
    DirPtrs D;
    float* phiu;
    const int* steps_left;  // the member's entry of the device table
    int tiles_x, tiles_y, chunk, items;
};
constexpr int kGridMembers = (32000 - 16) / (int)sizeof(GridMember);
struct BatchGrid {
    int n;
    GridMember m[kGridMembers];
};
static_assert(sizeof(BatchGrid) <= 32764, "kernel parameter space");

__global__ void __launch_bounds__(NT, LBMP_FUSED_MINB) step_batchg3_kernel(const __grid_constant__ BatchGrid G)
{
    extern __shared__ float smem[];
    const GridMember& M = G.m[blockIdx.y];
    if ((int)blockIdx.x >= M.items || *M.steps_left <= 0) return;  // spare CTA, or the member has finished
    const ThreadGeo T = thread_geo();
    const int tiles = M.tiles_x * M.tiles_y;
    for (int item = blockIdx.x; item < M.items; item += gridDim.x) {
        const int tile = item % tiles;
        const int z0 = M.p.zb + (item / tiles) * M.chunk;
        fused_segment(M.p, M.D, T, smem, (tile % M.tiles_x) * TX, (tile / M.tiles_x) * TY, z0,
                      min(z0 + M.chunk, M.p.ze), M.phiu);
    }
}

struct LaunchCfg {
    int device = -1;
    int per_sm = 0, sms = 0;
};
LaunchCfg g_cfg;

}  // namespace

#if LBMP_FUSED3_WITH_COMMON
// every domain has a fused kernel (FP32 and shifted 16-bit, D3Q27 and D2Q9,
// full and reduced phase lattice) but the divergence-term variant, which
// runs the reference pair
bool fused_supported(const lbmp_handle* h) { return !h->divu; }

__global__ void batch_epilogue_kernel(BatchDomain* table, int ndom)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d < ndom && table[d].steps_left > 0) {
        table[d].parity ^= 1;
        table[d].steps_left -= 1;
        table[d].p.step += 1;  // seeds the stochastic rounding of the next step's codes
    }
}

cudaError_t launch_batch_epilogue(BatchDomain* table, int ndom, cudaStream_t stream)
{
    if (ndom <= 0) return cudaSuccess;
    batch_epilogue_kernel<<<(ndom + 127) / 128, 128, 0, stream>>>(table, ndom);
    return cudaGetLastError();
}
#endif

namespace {

int g_batch_dev = -1;

// attributes of the batch kernel (not capturable: call before capture)
cudaError_t prepare_batch(int device)
{
    if (g_batch_dev != device) {
        const cudaError_t e =
            cudaFuncSetAttribute(step_batchg3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        g_batch_dev = device;
    }
    return cudaSuccess;
}

cudaError_t launch_batch_grid(const BatchDomain* host, const BatchDomain* dev, int n, int flip, int device,
                              cudaStream_t stream)
{
    if (g_batch_dev != device) return cudaErrorNotReady;  // prepare first
    if (n <= 0) return cudaSuccess;
    if (n > kGridMembers) return cudaErrorInvalidValue;
    BatchGrid G;
    memset(&G, 0, sizeof G);
    G.n = n;
    int xmax = 0;
    for (int k = 0; k < n; ++k) {
        const BatchDomain& B = host[k];
        GridMember& M = G.m[k];
        M.p = B.p;
        const int par = B.parity ^ flip;
        for (int a = 0; a < Q3; ++a) {
            const size_t off = (size_t)a * (size_t)B.p.N;
            M.D.fin[a] = B.f[par] + off;
            M.D.fout[a] = B.f[par ^ 1] + off;
        }
        for (int r = 0; r < QG; ++r) {
            const size_t off = (size_t)r * (size_t)B.p.N;
            M.D.gin[r] = B.g[par] + off;
            M.D.gout[r] = B.g[par ^ 1] + off;
        }
        M.phiu = B.phiu;
        M.steps_left = &dev[k].steps_left;
        M.tiles_x = B.tiles_x;
        M.tiles_y = B.tiles_y;
        M.chunk = B.chunk;
        M.items = B.items;
        xmax = B.items > xmax ? B.items : xmax;
    }
    if (xmax == 0) return cudaSuccess;
    const int gx = xmax < 65535 ? xmax : 65535;  // larger members loop over their items
    step_batchg3_kernel<<<dim3((unsigned)gx, (unsigned)n), NT, kSmemBytes, stream>>>(G);
    return cudaGetLastError();
}

}  // namespace

const Batch3Ops LBMP_BATCH3_OPS = {TX, TY, prepare_batch, nullptr, launch_batch_grid, kGridMembers};

cudaError_t LBMP_FUSED3_LAUNCH(lbmp_handle* h)
{
    if (g_cfg.device != h->device) {
        cudaError_t e = cudaFuncSetAttribute(step_fused3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemBytes);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_fused3_kernel, NT, kSmemBytes);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        if (e != cudaSuccess) return e;
        g_cfg.per_sm = per_sm > 0 ? per_sm : 1;
        g_cfg.sms = sms;
        g_cfg.device = h->device;
    }
    DirPtrs D;
    const int s = h->parity, d = 1 - h->parity;
    for (int a = 0; a < Q3; ++a) {
        const size_t off = (size_t)a * (size_t)h->N;
        D.fin[a] = h->f[s] + off;
        D.fout[a] = h->f[d] + off;
    }
    for (int r = 0; r < QG; ++r) {
        const size_t off = (size_t)r * (size_t)h->N;
        D.gin[r] = h->g[s] + off;
        D.gout[r] = h->g[d] + off;
    }
    FusedArgs A;
    A.phiu = h->phiu;
    A.tiles_x = (h->grid.nx + TX - 1) / TX;
    A.tiles_y = (h->grid.ny + TY - 1) / TY;
    const LaunchShape L = launch_shape(h, A.tiles_x * A.tiles_y, h->dp.ze - h->dp.zb, g_cfg.per_sm, g_cfg.sms);
    A.chunk = L.chunk;
    A.nitems = L.nitems;
    step_fused3_kernel<<<L.grid, NT, kSmemBytes, h->stream>>>(h->dp, A, D);
    return cudaGetLastError();
}

}  // namespace lbmp
