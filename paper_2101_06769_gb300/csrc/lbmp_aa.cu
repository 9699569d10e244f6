// lbmp_aa.cu -- the D3Q27 FP32 step on in-place AA storage (LBMP_FLAG_AA):
// one population set each for f' and g, updated in place, phi from a
// separate pass.
//
// Storage ("esoteric pull"): with the state in the natural phase the
// streamed value of direction a at cell x is A[a][x]; an even step reads
// those, collides, and writes the post-collision value of a to A[opp a][x],
// which leaves the state in the swapped phase: the streamed value of a at x
// is then A[opp a][x - c_a] (at a wall, A[a][x], the cell's own value bounced
// back).  An odd step reads those and writes the post-collision value of a
// to A[a][x + c_a] (across a wall, A[opp a][x]), which restores the natural
// phase.  In both steps every cell writes exactly the slots it read, so no
// two cells touch one slot and the update is race-free in place.
//
// phi = sum g is formed by the phase-aware phi pass of lbmp_kernels.cu
// before the step (the two-set kernels form it from the g they stage, ring
// cells included; here a ring cell's slots may already hold its owner's
// post-collision values).  The step stages phi of three planes (tile and
// ring) from that array and the tile's own g one plane ahead; the per-cell
// arithmetic is that of the two-set kernels (phase-field outputs first, the
// moment differences parked in the consumed g column), so the results equal
// them to within the rounding of separately compiled units.
#define LBMP_TILE_NS tile_aa
#define LBMP_FUSED_MINB 3
#define LBMP_OUT_ORDERED 1
#include "lbmp_internal.h"
#include "lbmp_tile.cuh"

namespace lbmp {

namespace {

using namespace tile_aa;

struct AAPtrs {
    float* f[Q3];  // per-direction bases of the single f' set
    float* g[Q3];  // and of the single g set
};

struct AAArgs {
    int tiles_x, tiles_y, chunk, nitems;
    const float* phi;  // phi hi [0, N), lo [N, 2N) from the phi pass
};

// slot holding the streamed value of direction a at cell (C, P)
template <bool Odd, bool Walls, int a>
__device__ __forceinline__ float* aa_src(float* const* base, const Column& C, const Plane& P)
{
    constexpr int cx = Lat<3>::cx(a), cy = Lat<3>::cy(a), cz = Lat<3>::cz(a);
    const int self = P.zs[1] + C.ys[1] + C.xs[1];
    if constexpr (!Odd) {
        return base[a] + self;
    } else {
        if (Walls && ((cz == 1 && P.lo) || (cz == -1 && P.hi))) return base[a] + self;
        return base[Lat<3>::opp(a)] + (P.zs[cz + 1] + C.ys[cy + 1] + C.xs[cx + 1]);
    }
}

// post-collision outputs: slot of the value of direction a after the step
template <bool Odd, bool Walls>
struct AAOut {
    static constexpr bool kTotal = false;
    float* const* base;
    const Column& C;
    const Plane& P;
    __device__ __forceinline__ void operator()(int a, float v) const
    {
        const int cx = Lat<3>::cx(a), cy = Lat<3>::cy(a), cz = Lat<3>::cz(a);
        const int self = P.zs[1] + C.ys[1] + C.xs[1];
        if (!Odd) {
            base[Lat<3>::opp(a)][self] = v;
        } else if (Walls && ((cz == -1 && P.lo) || (cz == 1 && P.hi))) {
            base[Lat<3>::opp(a)][self] = v;  // bounced back to the cell itself
        } else {
            base[a][P.zs[1 - cz] + C.ys[1 - cy] + C.xs[1 - cx]] = v;  // cell x + c_a
        }
    }
};

template <bool Odd, bool Walls>
struct AALoad {
    float* const* base;
    const Column& C;
    const Plane& P;
    float* v;
    template <int a>
    __device__ __forceinline__ void step() const
    {
        v[a] = *aa_src<Odd, Walls, a>(base, C, P);
    }
};

template <bool Odd, bool Walls>
struct AAStage {
    float* const* base;
    const Column& C;
    const Plane& P;
    float* buf;
    template <int a>
    __device__ __forceinline__ void step() const
    {
        cp_async4(buf + a * NT, aa_src<Odd, Walls, a>(base, C, P));
    }
};

// phi (hi, lo) of plane zz (mirrored beyond a wall) for the own and ring
// cells into one phi plane slot
__device__ __forceinline__ void stage_phi(const DevParams& p, const float* phi, const Column& own,
                                          const Column& ring, const ThreadGeo& T, int zz, float2* slot)
{
    const int pz = plane_src(p, zz);
    const long long base = (long long)pz * p.nx * p.ny;
    const long long io = base + own.ys[1] + own.xs[1];
    cp_async4(&slot[T.oslot].x, phi + io);
    cp_async4(&slot[T.oslot].y, phi + p.N + io);
    if (T.tid < NRING) {
        const long long ir = base + ring.ys[1] + ring.xs[1];
        cp_async4(&slot[T.rslot].x, phi + ir);
        cp_async4(&slot[T.rslot].y, phi + p.N + ir);
    }
}

template <bool Odd>
__device__ __forceinline__ void stage_g(const DevParams& p, const AAPtrs& D, const Column& own, int z, float* buf)
{
    Plane P;
    set_plane(P, p, z);
    if (P.lo || P.hi)
        Unroll<Q3>::run(AAStage<Odd, true>{D.g, own, P, buf});
    else
        Unroll<Q3>::run(AAStage<Odd, false>{D.g, own, P, buf});
}

template <bool Odd, bool Walls>
__device__ __forceinline__ void collide_cell(const DevParams& p, const AAPtrs& D, const Column& own, const Plane& P,
                                             const float2* pm, const float2* pc, const float2* pn, const FlowMoments& m,
                                             float* gcol)
{
    const float2 centre = pc[0];
    float grad[3], lap;
    stencil_from<3>(
        [&](int a) {
            const int cz = Lat<3>::cz(a);
            return (cz < 0 ? pm : (cz == 0 ? pc : pn))[Lat<3>::cy(a) * RX + Lat<3>::cx(a)];
        },
        centre, grad, lap);
    CellState s;
    float inv_rho, nu;
    flow_closure<3>(p, centre.x, grad, lap, m, s, inv_rho, nu);
    phase_outputs<3>(p, s, GFromStrided{gcol, NT}, centre.x, centre.y, AAOut<Odd, Walls>{D.g, own, P});
    float dh[27];
    flow_relax<3>(m, s, inv_rho, nu, dh);
#pragma unroll
    for (int a = 0; a < Q3; ++a) gcol[a * NT] = dh[a];
    flow_outputs<3>(s, DhStrided{gcol, NT}, m, AAOut<Odd, Walls>{D.f, own, P});
}

// planes [z0, z1) of the tile at (x0, y0); ends with a barrier
template <bool Odd>
__device__ __forceinline__ void aa_segment(const DevParams& p, const AAPtrs& D, const float* phi, const ThreadGeo& T,
                                           float* smem, int x0, int y0, int z0, int z1)
{
    float2* phiS = (float2*)smem;              // (hi, lo) [3][RY][RX]
    float* gS = (float*)(phiS + 3 * PLANE);    // [2][27][NT] own g, one plane ahead
    const int tid = T.tid;
    Column own, ring;
    set_column(own, p, pmod(x0 + T.tx, p.nx), pmod(y0 + T.ty, p.ny));
    set_column(ring, p, pmod(x0 + T.lx, p.nx), pmod(y0 + T.ly, p.ny));
    const bool valid = (x0 + T.tx < p.nx) && (y0 + T.ty < p.ny);
    int sP = 0, sC = 1, sN = 2;
    stage_phi(p, phi, own, ring, T, z0 - 1, phiS + sP * PLANE);
    stage_phi(p, phi, own, ring, T, z0, phiS + sC * PLANE);
    stage_g<Odd>(p, D, own, z0, gS + tid);
    cp_async_commit();
    for (int z = z0; z < z1; ++z) {
        const int cur = (z - z0) & 1;
        stage_phi(p, phi, own, ring, T, z + 1, phiS + sN * PLANE);
        cp_async_commit();  // group: phi of plane z+1 (needed now)
        if (z + 1 < z1) stage_g<Odd>(p, D, own, z + 1, gS + (cur ^ 1) * Q3 * NT + tid);
        cp_async_commit();  // group: g of plane z+1 (needed next iteration)
        Plane P;
        set_plane(P, p, z);
        float fr[Q3];
        if (P.lo || P.hi)
            Unroll<Q3>::run(AALoad<Odd, true>{D.f, own, P, fr});
        else
            Unroll<Q3>::run(AALoad<Odd, false>{D.f, own, P, fr});
        FlowMoments m;
        flow_moments<3>(m, fr);
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // all but the g of plane z+1
        __syncthreads();
        if (valid) {
            const float2* pm = phiS + sP * PLANE + T.oslot;
            const float2* pc = phiS + sC * PLANE + T.oslot;
            const float2* pn = phiS + sN * PLANE + T.oslot;
            float* gcol = gS + cur * Q3 * NT + tid;
            if (P.lo || P.hi)
                collide_cell<Odd, true>(p, D, own, P, pm, pc, pn, m, gcol);
            else
                collide_cell<Odd, false>(p, D, own, P, pm, pc, pn, m, gcol);
        }
        __syncthreads();  // phi slot and g buffer reuse
        const int t = sP;
        sP = sC;
        sC = sN;
        sN = t;
    }
    cp_async_wait_all();  // nothing of this segment is left in flight
}

constexpr size_t kSmemAA = sizeof(float2) * 3 * PLANE + sizeof(float) * 2 * Q3 * NT;

template <bool Odd>
__global__ void __launch_bounds__(NT, LBMP_FUSED_MINB) step_aa_kernel(DevParams p, AAArgs A, AAPtrs D)
{
    extern __shared__ float smem[];
    const ThreadGeo T = thread_geo();
    for (int item = blockIdx.x; item < A.nitems; item += gridDim.x) {
        const int tile = item % (A.tiles_x * A.tiles_y);
        const int chunk = item / (A.tiles_x * A.tiles_y);
        const int z0 = chunk * A.chunk;
        aa_segment<Odd>(p, D, A.phi, T, smem, (tile % A.tiles_x) * TX, (tile / A.tiles_x) * TY, z0,
                        min(z0 + A.chunk, p.nz));
    }
}

struct AACfg {
    int device = -1;
    int per_sm[2] = {0, 0}, sms = 0;
};
AACfg g_aa;

template <bool Odd>
cudaError_t launch_aa(lbmp_handle* h)
{
    if (g_aa.device != h->device) {
        for (int k = 0; k < 2; ++k) {
            const void* fn = k ? (const void*)step_aa_kernel<true> : (const void*)step_aa_kernel<false>;
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemAA);
            if (e != cudaSuccess) return e;
            int per = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, NT, kSmemAA);
            if (e != cudaSuccess) return e;
            g_aa.per_sm[k] = per > 0 ? per : 1;
        }
        cudaError_t e = cudaDeviceGetAttribute(&g_aa.sms, cudaDevAttrMultiProcessorCount, h->device);
        if (e != cudaSuccess) return e;
        g_aa.device = h->device;
    }
    AAPtrs D;
    for (int a = 0; a < Q3; ++a) {
        D.f[a] = h->f[0] + (size_t)a * (size_t)h->N;
        D.g[a] = h->g[0] + (size_t)a * (size_t)h->N;
    }
    AAArgs A;
    A.tiles_x = (h->grid.nx + TX - 1) / TX;
    A.tiles_y = (h->grid.ny + TY - 1) / TY;
    A.phi = h->phi;
    const LaunchShape L = launch_shape(h, A.tiles_x * A.tiles_y, h->grid.nz, g_aa.per_sm[Odd ? 1 : 0], g_aa.sms);
    A.chunk = L.chunk;
    A.nitems = L.nitems;
    step_aa_kernel<Odd><<<L.grid, NT, kSmemAA, h->stream>>>(h->dp, A, D);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_aa(lbmp_handle* h)
{
    // phi of the current state (phase-aware through dp.aa), then the step
    cudaError_t e = launch_phi_pass(h);
    if (e != cudaSuccess) return e;
    return h->parity ? launch_aa<true>(h) : launch_aa<false>(h);
}

}  // namespace lbmp
