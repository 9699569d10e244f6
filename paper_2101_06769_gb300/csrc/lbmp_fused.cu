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
// with the neighbouring tile's writes.  No phi field is stored, no separate
// phi pass runs; the only bytes beyond "every population read once and
// written once" are ring reads, which the neighbouring tiles fetch at about
// the same time (mostly L2 hits), and one extra plane per chunk.
//
// The per-cell arithmetic (lbmp_common.cuh) and the summation orders are the
// ones of the reference pair in lbmp_kernels.cu, so the two paths agree.
#include "lbmp_internal.h"

namespace lbmp {

namespace {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int RX = TX + 2, RY = TY + 2;
constexpr int NRING = 2 * RX + 2 * TY;
constexpr int Q3 = 27;
constexpr int PLANE = RY * RX;
constexpr size_t kSmemBytes = sizeof(float) * (2 * Q3 * NT + 2 * 3 * PLANE);

struct FusedArgs {
    const float* fin;
    const float* gin;
    float* fout;
    float* gout;
    int tiles_x, tiles_y, chunk, nchunks;
    int nitems;
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

// plane whose phi stands for plane zz: periodic wrap, or the mirrored ghost
// at a wall (reading A17)
__device__ __forceinline__ int plane_src(const DevParams& p, int zz)
{
    if (zz >= 0 && zz < p.nz) return zz;
    if (p.vert_periodic) return pmod(zz, p.nz);
    return zz < 0 ? 0 : p.nz - 1;
}

struct Geo {
    int tid, tx, ty, ox, oy;  // own column (wrapped for ragged tiles)
    int rx, ry, rslot;        // ring column (tid < NRING) and its smem slot
};

// phi on plane zz for the tile and its ring into phi_plane (hi at [0, PLANE),
// lo at [3 PLANE, 4 PLANE)); the tile's own g(zz) lands in gbuf (kept for the
// collision when zz is processed next).
__device__ __forceinline__ void stage_plane(const DevParams& p, const FusedArgs& A, const Geo& G, int zz,
                                            float* __restrict__ gbuf, float* __restrict__ phi_plane)
{
    const int zs = plane_src(p, zz);
    const long long self = ((long long)zs * p.ny + G.oy) * p.nx + G.ox;
#pragma unroll
    for (int a = 0; a < Q3; ++a) cp_async4(gbuf + a * NT + G.tid, A.gin + pull_index<3>(p, a, G.ox, G.oy, zs, self));
    cp_async_commit();
    if (G.tid < NRING) {
        const long long rself = ((long long)zs * p.ny + G.ry) * p.nx + G.rx;
        float v[Q3];
#pragma unroll
        for (int a = 0; a < Q3; ++a) v[a] = __ldg(A.gin + pull_index<3>(p, a, G.rx, G.ry, zs, rself));
        float hi = 0.f, lo = 0.f;
#pragma unroll
        for (int a = 0; a < Q3; ++a) phi_add(hi, lo, v[a]);
        phi_finish(hi, lo);
        phi_plane[G.rslot] = hi;
        phi_plane[3 * PLANE + G.rslot] = lo;
    }
    cp_async_wait_all();
    float hi = 0.f, lo = 0.f;
#pragma unroll
    for (int a = 0; a < Q3; ++a) phi_add(hi, lo, gbuf[a * NT + G.tid]);
    phi_finish(hi, lo);
    const int own = (G.ty + 1) * RX + (G.tx + 1);
    phi_plane[own] = hi;
    phi_plane[3 * PLANE + own] = lo;
}

__global__ void __launch_bounds__(NT, 2) step_fused3_kernel(DevParams p, FusedArgs A)
{
    extern __shared__ float smem[];
    float* gS = smem;                  // [2][27][NT]
    float* phiS = smem + 2 * Q3 * NT;  // hi [3][RY][RX], then lo [3][RY][RX]

    Geo G;
    G.tid = threadIdx.x;
    G.tx = G.tid % TX;
    G.ty = G.tid / TX;
    int lx = 0, ly = 0;
    if (G.tid < NRING) {
        const int r = G.tid;
        if (r < RX) {
            lx = r - 1;
            ly = -1;
        } else if (r < 2 * RX) {
            lx = r - RX - 1;
            ly = TY;
        } else if (r < 2 * RX + TY) {
            lx = -1;
            ly = r - 2 * RX;
        } else {
            lx = TX;
            ly = r - 2 * RX - TY;
        }
        G.rslot = (ly + 1) * RX + (lx + 1);
    }

    for (int item = blockIdx.x; item < A.nitems; item += gridDim.x) {
        const int tile = item % (A.tiles_x * A.tiles_y);
        const int chunk = item / (A.tiles_x * A.tiles_y);
        const int x0 = (tile % A.tiles_x) * TX, y0 = (tile / A.tiles_x) * TY;
        const int z0 = chunk * A.chunk;
        const int z1 = min(z0 + A.chunk, p.nz);
        G.ox = pmod(x0 + G.tx, p.nx);
        G.oy = pmod(y0 + G.ty, p.ny);
        const bool valid = (x0 + G.tx < p.nx) && (y0 + G.ty < p.ny);
        if (G.tid < NRING) {
            G.rx = pmod(x0 + lx, p.nx);
            G.ry = pmod(y0 + ly, p.ny);
        }
        int sP = 0, sC = 1, sN = 2;
        stage_plane(p, A, G, z0 - 1, gS + Q3 * NT, phiS + sP * PLANE);
        stage_plane(p, A, G, z0, gS, phiS + sC * PLANE);
        for (int z = z0; z < z1; ++z) {
            const int cur = (z - z0) & 1;
            const long long self = ((long long)z * p.ny + G.oy) * p.nx + G.ox;
            float fr[Q3];
#pragma unroll
            for (int a = 0; a < Q3; ++a) fr[a] = __ldg(A.fin + pull_index<3>(p, a, G.ox, G.oy, z, self));
            stage_plane(p, A, G, z + 1, gS + (cur ^ 1) * Q3 * NT, phiS + sN * PLANE);
            FlowMoments m;
            flow_moments<3>(m, fr);
            __syncthreads();
            if (valid) {
                float nh[Q3], nl[Q3];
#pragma unroll
                for (int a = 0; a < Q3; ++a) {
                    const int cz = Lat<3>::cz(a);
                    const float* pl = phiS + (cz < 0 ? sP : (cz == 0 ? sC : sN)) * PLANE;
                    const int o = (G.ty + 1 + Lat<3>::cy(a)) * RX + (G.tx + 1 + Lat<3>::cx(a));
                    nh[a] = pl[o];
                    nl[a] = pl[3 * PLANE + o];
                }
                float grad[3], lap;
                stencil_from_nb<3>(nh, nl, grad, lap);
                CellState s;
                float dh[27];
                flow_collide<3>(p, nh[13], grad, lap, m, s, dh);
                collide_outputs<3>(p, s, dh, m, GFromStrided{gS + cur * Q3 * NT + G.tid, NT}, nh[13], nl[13],
                                   SoAOut{A.fout + self, p.N}, SoAOut{A.gout + self, p.N});
            }
            __syncthreads();
            const int t = sP;
            sP = sC;
            sC = sN;
            sN = t;
        }
    }
}

struct LaunchCfg {
    int device = -1;
    int grid_cap = 0;
};
LaunchCfg g_cfg;

}  // namespace

bool fused_supported(const lbmp_handle* h) { return h->D == 3; }

cudaError_t launch_step_fused(lbmp_handle* h)
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
        g_cfg.grid_cap = (per_sm > 0 ? per_sm : 1) * sms;
        g_cfg.device = h->device;
    }
    FusedArgs A;
    const int s = h->parity, d = 1 - h->parity;
    A.fin = h->f[s];
    A.gin = h->g[s];
    A.fout = h->f[d];
    A.gout = h->g[d];
    A.tiles_x = (h->grid.nx + TX - 1) / TX;
    A.tiles_y = (h->grid.ny + TY - 1) / TY;
    const int tiles = A.tiles_x * A.tiles_y;
    // chunk length: enough items to balance the persistent grid, at least 8 planes
    int chunk = h->grid.nz;
    while (chunk > 8 && (long long)tiles * ((h->grid.nz + chunk - 1) / chunk) < 4LL * g_cfg.grid_cap) chunk /= 2;
    A.chunk = chunk;
    A.nchunks = (h->grid.nz + chunk - 1) / chunk;
    A.nitems = tiles * A.nchunks;
    const int grid = A.nitems < g_cfg.grid_cap ? A.nitems : g_cfg.grid_cap;
    step_fused3_kernel<<<grid, NT, kSmemBytes, h->stream>>>(h->dp, A);
    return cudaGetLastError();
}

}  // namespace lbmp
