// lbmp_fused2.cu -- fused single-pass D2Q9 step (and its batch form).
//
// The 2-D counterpart of lbmp_fused.cu: a CTA owns a segment of TX2 cells of
// one row and marches through a chunk of rows.  For row y it needs phi on rows
// y-1, y, y+1 over the segment and one cell on each side; phi = sum_a g_a of
// the pulled g, formed while g(y+1) is staged into shared memory by cp.async
// (the two side cells by threads 0 and 1).  The step reads one population
// set and writes the other, so the side reads never race with the
// neighbouring segment's writes.  The per-cell arithmetic is the shared one
// of lbmp_common.cuh, as in the reference pair.  Templated on PR, the phase
// field on the reduced lattice D2Q5 (first-order equilibrium and correction
// term, Sec. 2.2): 5 staged g values, and the stored previous phi u of the
// staged row copied with them.
#include "lbmp_internal.h"

namespace lbmp {

namespace {

constexpr int TX2 = 128;
constexpr int Q2 = 9;
constexpr int RW = TX2 + 2;  // row of phi incl. one side cell each way
// g of two rows, side cells, and (reduced phase lattice) phi u of two rows
constexpr size_t kSmem2 = sizeof(float) * (2 * Q2 * TX2 + Q2 * 2 + 2 * 2 * TX2) + sizeof(float2) * 4 * RW;

struct DirPtrs2 {
    const float* fin[Q2];
    const float* gin[Q2];
    float* fout[Q2];
    float* gout[Q2];
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

// 1: column and row offsets held as unsigned byte offsets (a pulled or
// stored address is the array base plus one 32-bit sum; arrays below
// 4 GiB); 0: signed element indices scaled to 64 bits at every access
#ifndef LBMP_F2_BYTEOFF
#define LBMP_F2_BYTEOFF 1
#endif
#if LBMP_F2_BYTEOFF
using off2 = unsigned;
constexpr unsigned kUnit2 = 4;
#else
using off2 = int;
constexpr int kUnit2 = 1;
#endif
__device__ __forceinline__ const float* at2(const float* base, off2 o)
{
    if constexpr (LBMP_F2_BYTEOFF != 0)
        return reinterpret_cast<const float*>(reinterpret_cast<const char*>(base) + o);
    else
        return base + o;
}
__device__ __forceinline__ int elem2(off2 o) { return (int)(o / kUnit2); }

// stores of one cell's outputs (per-direction array bases, one cell offset)
struct Out2 {
    static constexpr bool kTotal = false;
    float* const* base;
    off2 self;
    __device__ __forceinline__ void operator()(int a, float v) const { *const_cast<float*>(at2(base[a], self)) = v; }
};

// upstream x coordinates xs[c+1] = x - c (periodic); with a symmetry x axis
// (reading A28) the column's own neighbours, clamped, and slo / shi flag the
// columns next to the left / right symmetry face
struct Col2 {
    off2 xs[3];
    bool slo, shi;
};
__device__ __forceinline__ void set_col2(Col2& C, int x, int nx)
{
    C.xs[0] = (off2)(x + 1 == nx ? 0 : x + 1) * kUnit2;
    C.xs[1] = (off2)x * kUnit2;
    C.xs[2] = (off2)(x == 0 ? nx - 1 : x - 1) * kUnit2;
    C.slo = C.shi = false;
}
__device__ __forceinline__ void set_col2_sym(Col2& C, int x, int nx)
{
    C.xs[0] = (off2)(x + 1 == nx ? x : x + 1) * kUnit2;
    C.xs[1] = (off2)x * kUnit2;
    C.xs[2] = (off2)(x == 0 ? 0 : x - 1) * kUnit2;
    C.slo = x == 0;
    C.shi = x == nx - 1;
}
// column x of the lattice or its mirror image across a symmetry face (clamped:
// the columns further out than the first ghost feed no stencil)
__device__ __forceinline__ int reflect_col(int x, int nx)
{
    const int r = x < 0 ? -1 - x : (x >= nx ? 2 * nx - 1 - x : x);
    return r < 0 ? 0 : (r >= nx ? nx - 1 : r);
}

// upstream rows ys[c+1] = (y - c) nx; lo/hi: bottom/top row of a walled domain
struct Row2 {
    off2 ys[3];
    bool lo, hi;
};
__device__ __forceinline__ void set_row2(Row2& R, const DevParams& p, int y)
{
    R.lo = !p.vert_periodic && y == 0;
    R.hi = !p.vert_periodic && y == p.ny - 1;
    R.ys[0] = (off2)((y + 1 == p.ny ? 0 : y + 1) * p.nx) * kUnit2;
    R.ys[1] = (off2)(y * p.nx) * kUnit2;
    R.ys[2] = (off2)((y == 0 ? p.ny - 1 : y - 1) * p.nx) * kUnit2;
}

// post-streaming population a of the cell (C, R): pulled from upstream,
// bounced back at a wall, or (SX) reflected at a symmetry face: the value
// that left the cell's own column, one row upstream, with the mirrored x
// velocity
template <bool SX>
__device__ __forceinline__ const float* pulled2(const float* const* base, int a, const Col2& C, const Row2& R)
{
    const int cx = Lat<2>::cx(a), cy = Lat<2>::cy(a);
    if ((cy == 1 && R.lo) || (cy == -1 && R.hi)) return at2(base[Lat<2>::opp(a)], R.ys[1] + C.xs[1]);
    if (SX && ((cx == 1 && C.slo) || (cx == -1 && C.shi))) return at2(base[Lat<2>::mx(a)], R.ys[cy + 1] + C.xs[1]);
    return at2(base[a], R.ys[cy + 1] + C.xs[cx + 1]);
}

// the same for slot r of the phase lattice (PR: D2Q5 slots, opposite QG-1-r)
// (a face population's mirror image is its opposite slot)
template <bool PR, bool SX>
__device__ __forceinline__ const float* pulled2_g(const float* const* base, int r, const Col2& C, const Row2& R)
{
    if constexpr (!PR) {
        return pulled2<SX>(base, r, C, R);
    } else {
        constexpr int QG = PhaseLat<2, true>::Q;
        const int a = PhaseLat<2, true>::full(r);
        const int cx = Lat<2>::cx(a), cy = Lat<2>::cy(a);
        if ((cy == 1 && R.lo) || (cy == -1 && R.hi)) return at2(base[QG - 1 - r], R.ys[1] + C.xs[1]);
        if (SX && ((cx == 1 && C.slo) || (cx == -1 && C.shi))) return at2(base[QG - 1 - r], R.ys[1] + C.xs[1]);
        return at2(base[r], R.ys[cy + 1] + C.xs[cx + 1]);
    }
}

__device__ __forceinline__ int row_src(const DevParams& p, int yy)
{
    if (yy >= 0 && yy < p.ny) return yy;
    if (p.vert_periodic) return pmod(yy, p.ny);
    return yy < 0 ? 0 : p.ny - 1;  // mirrored ghost (reading A17)
}

// stage row yy: own g into gbuf, side cells' g into sbuf, then phi into
// prow; PR: also the own cells' stored phi u of that row into ubuf [2][TX2]
template <bool PR, bool SX>
__device__ __forceinline__ void stage_row(const DevParams& p, const DirPtrs2& D, const Col2& own, const Col2& side,
                                          int tid, int yy, float* __restrict__ gbuf, float* __restrict__ sbuf,
                                          float2* __restrict__ prow, const float* __restrict__ phiu,
                                          float* __restrict__ ubuf)
{
    constexpr int QG = PhaseLat<2, PR>::Q;
    Row2 R;
    set_row2(R, p, row_src(p, yy));
#pragma unroll
    for (int r = 0; r < QG; ++r) cp_async4(gbuf + r * TX2 + tid, pulled2_g<PR, SX>(D.gin, r, own, R));
    if (tid < 2) {
#pragma unroll
        for (int r = 0; r < QG; ++r) cp_async4(sbuf + r * 2 + tid, pulled2_g<PR, SX>(D.gin, r, side, R));
    }
    if constexpr (PR) {
        const int self = elem2(R.ys[1] + own.xs[1]);
        cp_async4(ubuf + tid, phiu + self);
        cp_async4(ubuf + TX2 + tid, phiu + p.N + self);
    }
    cp_async_commit();
    cp_async_wait_all();
    float hi, lo;
    if (tid < 2) {
        phi_sum_phase<2, PR>([&](int r) { return sbuf[r * 2 + tid]; }, hi, lo);
        prow[tid == 0 ? 0 : RW - 1] = make_float2(hi, lo);
    }
    phi_sum_phase<2, PR>([&](int r) { return gbuf[r * TX2 + tid]; }, hi, lo);
    prow[tid + 1] = make_float2(hi, lo);
}

// rows [y0, y1) of the segment starting at x0.  One barrier per row: every
// shared value but phi is written and read by the same thread, and phi of
// row yy sits in slot (yy - y0 + 1) & 3 of four, so the row staged in an
// iteration is never one that a slower thread still reads from the previous
// one (a thread is at most one iteration ahead: it must pass that
// iteration's barrier first).  Ends with a barrier, so the caller may reuse
// shared memory afterwards.
// SXM: kSymOff (periodic x) or kSymOn (x a symmetry axis)
constexpr int kSymOff = 0, kSymOn = 1;
template <bool PR, int SXM>
__device__ __forceinline__ void fused2_segment(const DevParams& p, const DirPtrs2& D, float* smem, int x0, int y0,
                                               int y1, float* __restrict__ phiu)
{
    constexpr int QG = PhaseLat<2, PR>::Q;
    float* gS = smem;                               // [2][QG][TX2]
    float* sS = smem + 2 * Q2 * TX2;                // [QG][2]
    float2* phiS = (float2*)(sS + Q2 * 2);          // [4][RW]
    float* uS = (float*)(phiS + 4 * RW);            // [2][2][TX2] phi u (PR)
    const int tid = threadIdx.x;
    Col2 own, side;
    constexpr bool SX = SXM != kSymOff;
    if (SXM == kSymOn) {
        // ghost columns mirror the boundary columns instead of wrapping
        set_col2_sym(own, reflect_col(x0 + tid, p.nx), p.nx);
        set_col2_sym(side, reflect_col(tid == 0 ? x0 - 1 : x0 + TX2, p.nx), p.nx);
    } else {
        set_col2(own, pmod(x0 + tid, p.nx), p.nx);
        set_col2(side, pmod(tid == 0 ? x0 - 1 : x0 + TX2, p.nx), p.nx);
    }
    const bool valid = x0 + tid < p.nx;
    stage_row<PR, SX>(p, D, own, side, tid, y0 - 1, gS + QG * TX2, sS, phiS, phiu, uS + 2 * TX2);
    stage_row<PR, SX>(p, D, own, side, tid, y0, gS, sS, phiS + RW, phiu, uS);
    for (int y = y0; y < y1; ++y) {
        const int cur = (y - y0) & 1;
        const int sP = (y - y0) & 3, sC = (y - y0 + 1) & 3, sN = (y - y0 + 2) & 3;
        Row2 R;
        set_row2(R, p, y);
        float fr[Q2];
#pragma unroll
        for (int a = 0; a < Q2; ++a) fr[a] = __ldg(pulled2<SX>(D.fin, a, own, R));
        stage_row<PR, SX>(p, D, own, side, tid, y + 1, gS + (cur ^ 1) * QG * TX2, sS, phiS + sN * RW, phiu,
                      uS + (cur ^ 1) * 2 * TX2);
        FlowMoments m;
        flow_moments<2>(m, fr);
        __syncthreads();
        if (valid) {
            float nh[Q2], nl[Q2];
#pragma unroll
            for (int a = 0; a < Q2; ++a) {
                const int cy = Lat<2>::cy(a);
                const float2 v = phiS[(cy < 0 ? sP : (cy == 0 ? sC : sN)) * RW + tid + 1 + Lat<2>::cx(a)];
                nh[a] = v.x;
                nl[a] = v.y;
            }
            float grad[3], lap;
            stencil_from_nb<2>(nh, nl, grad, lap);
            CellState s;
            float dh[27];
            flow_collide<2>(p, nh[4], grad, lap, m, s, dh);
            const off2 self = R.ys[1] + own.xs[1];
            if constexpr (PR)
                collide_outputs<2, true>(p, s, DhArray{dh}, m, GFromStrided{gS + cur * QG * TX2 + tid, TX2}, nh[4],
                                         nl[4], Out2{D.fout, self}, Out2{D.gout, self},
                                         PhiUStaged<2>{p, phiu, elem2(self), uS + cur * 2 * TX2 + tid, TX2});
            else
                collide_outputs<2>(p, s, DhArray{dh}, m, GFromStrided{gS + cur * Q2 * TX2 + tid, TX2}, nh[4], nl[4],
                                   Out2{D.fout, self}, Out2{D.gout, self});
        }
    }
    __syncthreads();
}

struct Fused2Args {
    int tiles_x, chunk, nitems;
    float* phiu;  // reduced phase lattice: stored previous phi u; else null
};

template <bool PR, bool SX>
__global__ void __launch_bounds__(TX2, 7) step_fused2_kernel(DevParams p, Fused2Args A, DirPtrs2 D)
{
    extern __shared__ float smem[];
    for (int item = blockIdx.x; item < A.nitems; item += gridDim.x) {
        const int tile = item % A.tiles_x;
        const int y0 = (item / A.tiles_x) * A.chunk;
        fused2_segment<PR, SX ? kSymOn : kSymOff>(p, D, smem, tile * TX2, y0, min(y0 + A.chunk, p.ny), A.phiu);
    }
}

template <bool PR, bool SX>
__global__ void __launch_bounds__(TX2) step_batch2_kernel(const BatchDomain* __restrict__ table, int ndom,
                                                          int nitems)
{
    extern __shared__ float smem[];
    __shared__ DevParams sp;
    __shared__ DirPtrs2 sd;
    __shared__ int s_dom, s_tx, s_chunk, s_begin, s_active;
    __shared__ float* s_phiu;
    int cur = -1;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int lo = 0, hi = ndom - 1;
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
                s_chunk = B.chunk;
                s_begin = B.item_begin;
                s_active = B.steps_left > 0;
                s_phiu = B.phiu;
            }
            const int par = B.parity;
            constexpr int QG = PhaseLat<2, PR>::Q;
            for (int k = threadIdx.x; k < 4 * Q2; k += blockDim.x) {
                const int set = k / Q2, a = k % Q2;
                const size_t off = (size_t)a * (size_t)B.p.N;
                if (set == 0) sd.fin[a] = B.f[par] + off;
                if (set == 1 && a < QG) sd.gin[a] = B.g[par] + off;
                if (set == 2) sd.fout[a] = B.f[par ^ 1] + off;
                if (set == 3 && a < QG) sd.gout[a] = B.g[par ^ 1] + off;
            }
            cur = d;
            __syncthreads();
        }
        if (!s_active) continue;
        const int local = item - s_begin;
        const int tile = local % s_tx;
        const int y0 = (local / s_tx) * s_chunk;
        fused2_segment<PR, SX ? kSymOn : kSymOff>(sp, sd, smem, tile * TX2, y0, min(y0 + s_chunk, sp.ny), s_phiu);
    }
}

// launch configuration per phase lattice and x boundary [PR + 2 SX] of the
// single-domain and of the batch kernel
int g_f2_dev[4] = {-1, -1, -1, -1}, g_f2_per_sm[4] = {0, 0, 0, 0}, g_f2_sms[4] = {0, 0, 0, 0},
    g_b2_dev[4] = {-1, -1, -1, -1}, g_b2_cap[4] = {0, 0, 0, 0};

cudaError_t setup_kernel(const void* fn, int device, int& dev_cached, int& per_sm_out, int& sms_out)
{
    if (dev_cached == device) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem2);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TX2, kSmem2);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    per_sm_out = per_sm > 0 ? per_sm : 1;
    sms_out = sms;
    dev_cached = device;
    return cudaSuccess;
}

}  // namespace

int batch2_tile_x() { return TX2; }

cudaError_t launch_step_fused2(lbmp_handle* h)
{
    const bool sx = h->dp.sym_x != 0;
    const int k = (h->reduced ? 1 : 0) + (sx ? 2 : 0);
    const void* fns[4] = {(const void*)step_fused2_kernel<false, false>, (const void*)step_fused2_kernel<true, false>,
                          (const void*)step_fused2_kernel<false, true>, (const void*)step_fused2_kernel<true, true>};
    cudaError_t e = setup_kernel(fns[k], h->device, g_f2_dev[k], g_f2_per_sm[k], g_f2_sms[k]);
    if (e != cudaSuccess) return e;
    DirPtrs2 D;
    const int s = h->parity, d = 1 - h->parity;
    for (int a = 0; a < Q2; ++a) {
        const size_t off = (size_t)a * (size_t)h->N;
        D.fin[a] = h->f[s] + off;
        D.fout[a] = h->f[d] + off;
        D.gin[a] = a < h->Qg ? h->g[s] + off : nullptr;
        D.gout[a] = a < h->Qg ? h->g[d] + off : nullptr;
    }
    Fused2Args A;
    A.tiles_x = (h->grid.nx + TX2 - 1) / TX2;
    const LaunchShape L = launch_shape(h, A.tiles_x, h->grid.ny, g_f2_per_sm[k], g_f2_sms[k]);
    A.chunk = L.chunk;
    A.nitems = L.nitems;
    A.phiu = h->phiu;
    switch (k) {
    case 0: step_fused2_kernel<false, false><<<L.grid, TX2, kSmem2, h->stream>>>(h->dp, A, D); break;
    case 1: step_fused2_kernel<true, false><<<L.grid, TX2, kSmem2, h->stream>>>(h->dp, A, D); break;
    case 2: step_fused2_kernel<false, true><<<L.grid, TX2, kSmem2, h->stream>>>(h->dp, A, D); break;
    default: step_fused2_kernel<true, true><<<L.grid, TX2, kSmem2, h->stream>>>(h->dp, A, D); break;
    }
    return cudaGetLastError();
}

cudaError_t prepare_batch2(int device, bool reduced, bool sym)
{
    const int k = (reduced ? 1 : 0) + (sym ? 2 : 0);
    const void* fns[4] = {(const void*)step_batch2_kernel<false, false>, (const void*)step_batch2_kernel<true, false>,
                          (const void*)step_batch2_kernel<false, true>, (const void*)step_batch2_kernel<true, true>};
    int per_sm = 0, sms = 0, dev = g_b2_dev[k];
    cudaError_t e = setup_kernel(fns[k], device, dev, per_sm, sms);
    if (e == cudaSuccess && g_b2_dev[k] != device) {
        g_b2_cap[k] = per_sm * sms;
        g_b2_dev[k] = device;
    }
    return e;
}

cudaError_t launch_batch2(const BatchDomain* table, int ndom, int nitems, int device, cudaStream_t stream,
                          bool reduced, bool sym)
{
    const int k = (reduced ? 1 : 0) + (sym ? 2 : 0);
    if (g_b2_dev[k] != device) return cudaErrorNotReady;  // prepare_batch2 first
    if (nitems <= 0) return cudaSuccess;
    const int grid = nitems < g_b2_cap[k] ? nitems : g_b2_cap[k];
    switch (k) {
    case 0: step_batch2_kernel<false, false><<<grid, TX2, kSmem2, stream>>>(table, ndom, nitems); break;
    case 1: step_batch2_kernel<true, false><<<grid, TX2, kSmem2, stream>>>(table, ndom, nitems); break;
    case 2: step_batch2_kernel<false, true><<<grid, TX2, kSmem2, stream>>>(table, ndom, nitems); break;
    default: step_batch2_kernel<true, true><<<grid, TX2, kSmem2, stream>>>(table, ndom, nitems); break;
    }
    return cudaGetLastError();
}

}  // namespace lbmp
