// lbmp_fused2s.cu -- fused single-pass D2Q9 step for the shifted 16-bit
// storage forms (and its batch form).
//
// The work decomposition of the FP32 D2Q9 kernel (lbmp_fused2.cu): a CTA owns
// a segment of TX2 cells of one row and marches through a chunk of rows; phi
// of rows y-1, y, y+1 over the segment and one side cell each way lives in
// shared memory.  A pulled value needs its 16-bit code and the FP32 reference
// R of the cell that wrote it.  As in the 3-D 16-bit kernel
// (lbmp_fused16.cu), the writers' references are staged by cp.async in
// shared memory, one new row per population set and iteration: f' over the
// segment and one side cell each way, g over the segment and two (a side
// cell's phi pulls from one cell further out).  The codes are loaded to
// registers (2-byte loads, 32-bit cell offsets from per-direction array
// bases).  Each thread decodes its own cell's pulled g of row y+1 (threads 0
// and 1 the two side cells as well), sums phi from the exact parts of the
// values (phi_sum_shifted) and keeps the decoded own values for the
// collision.  Decoding, the collision and the encoding are those of the
// reference pair (lbmp_kernels.cu), in the same order.
#include <type_traits>

#include "lbmp_internal.h"

namespace lbmp {

namespace {

constexpr int TX2 = 128;
constexpr int Q2 = 9;
constexpr int C2 = 4;
constexpr int RW = TX2 + 2;  // row of phi and of f' references: segment plus one side cell each way
constexpr int GW = TX2 + 4;  // row of g references: segment plus two cells each way
constexpr int kRefRows = 8;  // reference rows per set in rotation (row k in slot k & 7)
constexpr size_t kSmem2s =
    sizeof(float) * (2 * Q2 * TX2 + kRefRows * (RW + GW)) + sizeof(float2) * 4 * RW;

struct DirPtrs2s {
    const unsigned short* fin[Q2];  // per-direction code arrays; entry C2 unused
    const unsigned short* gin[Q2];
    unsigned short* fout[Q2];
    unsigned short* gout[Q2];
    const float* rfin;  // references
    const float* rgin;
    float* rfout;
    float* rgout;
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

__device__ __forceinline__ bool ghost_row(const DevParams& p, int yy)
{
    return !p.vert_periodic && (yy < 0 || yy >= p.ny);
}

// reference row k (logical; periodic wrap) into slot k & 7 of rows of length
// L; entry e of the row holds column xa (e = tid) or xb (e = tid + TX2 < L).
// Rows beyond a wall are never read (their populations bounce) and are skipped.
__device__ __forceinline__ void load_ref_row(const DevParams& p, const float* src, int k, float* rows, int L, int xa,
                                             int xb, int tid)
{
    int yk = k;
    if (k < 0 || k >= p.ny) {
        if (!p.vert_periodic) return;
        yk = pmod(k, p.ny);
    }
    const float* base = src + yk * p.nx;
    float* d = rows + (k & (kRefRows - 1)) * L;
    cp_async4(d + tid, base + xa);
    if (tid + TX2 < L) cp_async4(d + tid + TX2, base + xb);
}

// columns x-1, x, x+1 (periodic) and rows y+1, y, y-1 (periodic, or flagged
// at a wall) of a cell, as offsets: index [c+1] is the upstream neighbour x - c
// 1: the offsets are unsigned byte offsets of the 2-byte codes (a pulled or
// stored code's address is its array base plus one 32-bit sum); 0: signed
// element indices scaled to 64 bits at every access
#ifndef LBMP_F2S_BYTEOFF
#define LBMP_F2S_BYTEOFF 1
#endif
#if LBMP_F2S_BYTEOFF
using off2s = unsigned;
constexpr unsigned kUnit2s = 2;
#else
using off2s = int;
constexpr int kUnit2s = 1;
#endif
template <class E>
__device__ __forceinline__ E* at2s(E* base, off2s o)
{
    if constexpr (LBMP_F2S_BYTEOFF != 0) {
        static_assert(sizeof(E) == 2, "byte offsets of the 2-byte codes");
        using B = typename std::conditional<std::is_const<E>::value, const char, char>::type;
        return reinterpret_cast<E*>(reinterpret_cast<B*>(base) + o);
    } else {
        return base + o;
    }
}
__device__ __forceinline__ int elem2s(off2s o) { return (int)(o / kUnit2s); }

struct Cell2 {
    off2s xs[3], ys[3];
    bool lo, hi;
};

__device__ __forceinline__ void set_cell2(Cell2& C, const DevParams& p, int x, int y)
{
    C.xs[0] = (off2s)(x + 1 == p.nx ? 0 : x + 1) * kUnit2s;
    C.xs[1] = (off2s)x * kUnit2s;
    C.xs[2] = (off2s)(x == 0 ? p.nx - 1 : x - 1) * kUnit2s;
    C.lo = !p.vert_periodic && y == 0;
    C.hi = !p.vert_periodic && y == p.ny - 1;
    C.ys[0] = (off2s)((y + 1 == p.ny ? 0 : y + 1) * p.nx) * kUnit2s;
    C.ys[1] = (off2s)(y * p.nx) * kUnit2s;
    C.ys[2] = (off2s)((y == 0 ? p.ny - 1 : y - 1) * p.nx) * kUnit2s;
}

// the encoder of one cell's outputs (as EncPtr) at a cell offset: the codes
// at base + offset, the reference at its 4-byte slot
template <class St>
struct EncCell2 {
    static constexpr bool kTotal = true;
    unsigned short* const* qb;
    float* R;
    off2s self;
    float off;
    mutable float sq;
    unsigned seed;  // code_seed of the writer cell (stochastic rounding)
    __device__ __forceinline__ void operator()(int a, float v) const
    {
        const float W = wint<2>(a);
        const unsigned short c = enc_code<St>(fmaf(v, St::S / W, -off), seed, a);
        *at2s(qb[a], self) = c;
        sq += St::dec(c) * (W * St::s);
    }
    __device__ __forceinline__ void finish(float th, float tl) const
    {
        R[elem2s(self)] = ref_from_total<2>(th, tl, sq);
    }
};

// code of the pulled population a of cell C, and whether it bounced at a wall
// (then it is the opposite population of the cell itself); a is a
// compile-time constant at every (unrolled) call site
__device__ __forceinline__ unsigned short pulled_code(const unsigned short* const* q, int a, const Cell2& C,
                                                      bool& bounced)
{
    const int cx = Lat<2>::cx(a), cy = Lat<2>::cy(a);
    bounced = (cy == 1 && C.lo) || (cy == -1 && C.hi);
    if (bounced) return __ldg(at2s(q[Lat<2>::opp(a)], C.ys[1] + C.xs[1]));
    return __ldg(at2s(q[a], C.ys[cy + 1] + C.xs[cx + 1]));
}

// Decode the pulled g of one cell of row yy and sum its phi (hi, lo); Keep:
// also store the decoded values (= wr + wq, rounded once) at buf[a * TX2].
// yy is a logical row (y0 - 1 .. y1; not a ghost row beyond a wall): the
// codes are read from its periodic image, the references from the slots of
// the logical rows yy-1, yy, yy+1 in RG; e is the cell's entry in a
// reference row.
template <class St, bool Keep>
__device__ __forceinline__ float2 decode_g_cell(const DevParams& p, const DirPtrs2s& D, const float* RG, int yy,
                                                int x, int e, float* buf)
{
    Cell2 C;
    set_cell2(C, p, x, pmod(yy, p.ny));
    const float* R0 = RG + (yy & (kRefRows - 1)) * GW + e;
    float hi, lo;
    phi_sum_shifted<2>(
        [&](int a, float& wr, float& wq) {
            const float W = wint<2>(a);
            if (a == C2) {
                wr = W * R0[0];
                wq = 0.f;
                if (Keep) buf[a * TX2] = wr;
                return;
            }
            bool bounced;
            const unsigned short c = pulled_code(D.gin, a, C, bounced);
            const int cx = Lat<2>::cx(a), cy = Lat<2>::cy(a);
            const float R = bounced ? R0[0] : RG[((yy - cy) & (kRefRows - 1)) * GW + e - cx];
            const float qv = St::dec(c);
            wr = W * R;
            wq = qv * (W * St::s);
            if (Keep) buf[a * TX2] = dec_value<2, St>(a, qv, R);
        },
        hi, lo);
    return make_float2(hi, lo);
}

// rows [y0, y1) of the segment starting at x0.  One barrier per row: the
// decoded g is private to its thread; phi of row yy sits in slot
// (yy - y0 + 1) & 3 of four and the references of row k in slot k & 7 of
// eight, so what an iteration stages is never what a slower thread still
// reads from the previous one (a thread is at most one iteration ahead: it
// must pass that iteration's barrier first).  Ends with a barrier, so the
// caller may reuse shared memory afterwards.
template <class St>
__device__ __forceinline__ void fused2s_segment(const DevParams& p, const DirPtrs2s& D, float* smem, int x0, int y0,
                                                int y1)
{
    float* gS = smem;                          // [2][9][TX2] decoded g of the staged rows
    float* RF = gS + 2 * Q2 * TX2;             // [8][RW] f' references
    float* RG = RF + kRefRows * RW;            // [8][GW] g references
    float2* phiS = (float2*)(RG + kRefRows * GW);  // [4][RW]
    const int tid = threadIdx.x;
    const int x_own = pmod(x0 + tid, p.nx);
    const int x_side = pmod(tid == 0 ? x0 - 1 : x0 + TX2, p.nx);
    const int e_side = tid == 0 ? 1 : TX2 + 2;  // side cell's entry in a g reference row
    const bool valid = x0 + tid < p.nx;
    const int fa = pmod(x0 - 1 + tid, p.nx), fb = pmod(x0 - 1 + tid + TX2, p.nx);
    const int ga = pmod(x0 - 2 + tid, p.nx), gb = pmod(x0 - 2 + tid + TX2, p.nx);
    // decode g of row yy (own cell into gbuf, side cells for tid < 2) and write
    // its phi into slot ps; a ghost row beyond a wall copies the wall row's phi
    // from slot pw (each thread the entries it writes itself)
    const auto stage_g = [&](int yy, float* gbuf, int ps, int pw) {
        float2* prow = phiS + ps * RW;
        if (ghost_row(p, yy)) {
            const float2* wrow = phiS + pw * RW;
            if (tid < 2) prow[tid == 0 ? 0 : RW - 1] = wrow[tid == 0 ? 0 : RW - 1];
            prow[tid + 1] = wrow[tid + 1];
            return;
        }
        if (tid < 2) prow[tid == 0 ? 0 : RW - 1] = decode_g_cell<St, false>(p, D, RG, yy, x_side, e_side, nullptr);
        prow[tid + 1] = decode_g_cell<St, true>(p, D, RG, yy, x_own, tid + 2, gbuf + tid);
    };
    // references for the first rows: g rows y0-2 .. y0+2, f' rows y0-1 .. y0+1
    for (int k = y0 - 2; k <= y0 + 2; ++k) load_ref_row(p, D.rgin, k, RG, GW, ga, gb, tid);
    for (int k = y0 - 1; k <= y0 + 1; ++k) load_ref_row(p, D.rfin, k, RF, RW, fa, fb, tid);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    if (ghost_row(p, y0 - 1)) {  // the wall row first, then its mirror
        stage_g(y0, gS, 1, 0);
        stage_g(y0 - 1, gS + Q2 * TX2, 0, 1);
    } else {
        stage_g(y0 - 1, gS + Q2 * TX2, 0, 0);
        stage_g(y0, gS, 1, 0);
    }
    for (int y = y0; y < y1; ++y) {
        const int cur = (y - y0) & 1;
        const int sP = (y - y0) & 3, sC = (y - y0 + 1) & 3, sN = (y - y0 + 2) & 3;
        // references of the rows the next iteration adds, in flight during this one
        load_ref_row(p, D.rgin, y + 3, RG, GW, ga, gb, tid);
        load_ref_row(p, D.rfin, y + 2, RF, RW, fa, fb, tid);
        cp_async_commit();
        Cell2 C;
        set_cell2(C, p, x_own, y);
        unsigned short q[Q2];
        bool bq[Q2];
#pragma unroll
        for (int a = 0; a < Q2; ++a)
            if (a != C2) q[a] = pulled_code(D.fin, a, C, bq[a]);
        stage_g(y + 1, gS + (cur ^ 1) * Q2 * TX2, sN, sC);
        FlowMoments m;
        {
            const float* R0 = RF + (y & (kRefRows - 1)) * RW + tid + 1;
            float fr[Q2];
#pragma unroll
            for (int a = 0; a < Q2; ++a) {
                const int cx = Lat<2>::cx(a), cy = Lat<2>::cy(a);
                if (a == C2) {
                    fr[a] = wint<2>(C2) * R0[0];
                } else {
                    const float R = bq[a] ? R0[0] : RF[((y - cy) & (kRefRows - 1)) * RW + tid + 1 - cx];
                    fr[a] = dec_value<2, St>(a, St::dec(q[a]), R);
                }
            }
            flow_moments<2>(m, fr);
        }
        cp_async_wait_all();
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
            flow_collide<2>(p, nh[C2], grad, lap, m, s, dh);
            const off2s self = C.ys[1] + C.xs[1];
            const GFromStrided gi{gS + cur * Q2 * TX2 + tid, TX2};
            float off_f, off_g;
            rest_offsets<2, St>(p, s, dh, gi, off_f, off_g);
            const EncCell2<St> fo{D.fout, D.rfout, self, off_f, 0.f, code_seed(p, elem2s(self), 0)};
            const EncCell2<St> go{D.gout, D.rgout, self, off_g, 0.f, code_seed(p, elem2s(self), 1)};
            collide_outputs<2>(p, s, DhArray{dh}, m, gi, nh[C2], nl[C2], fo, go);
        }
    }
    __syncthreads();
}

struct Fused2sArgs {
    int tiles_x, chunk, nitems;
};

template <class St>
__global__ void __launch_bounds__(TX2, 6) step_fused2s_kernel(DevParams p, Fused2sArgs A, DirPtrs2s D)
{
    extern __shared__ __align__(16) float smem2s[];
    for (int item = blockIdx.x; item < A.nitems; item += gridDim.x) {
        const int tile = item % A.tiles_x;
        const int y0 = (item / A.tiles_x) * A.chunk;
        fused2s_segment<St>(p, D, smem2s, tile * TX2, y0, min(y0 + A.chunk, p.ny));
    }
}

// direction bases of population sets f (in, out) and g (in, out) of parity par
__host__ __device__ inline void dir_ptrs2s(DirPtrs2s& D, float* const f[2], float* const g[2], int par, long long N,
                                           int k)
{
    const int set = k / Q2, a = k % Q2;
    const size_t off = (size_t)(a - (a > C2)) * (size_t)N;
    unsigned short* base = (unsigned short*)((set == 0 || set == 2 ? f : g)[set < 2 ? par : par ^ 1] + N);
    unsigned short* q = a != C2 ? base + off : nullptr;
    if (set == 0) D.fin[a] = q;
    if (set == 1) D.gin[a] = q;
    if (set == 2) D.fout[a] = q;
    if (set == 3) D.gout[a] = q;
}

template <class St>
__global__ void __launch_bounds__(TX2) step_batch2s_kernel(const BatchDomain* __restrict__ table, int ndom,
                                                           int nitems)
{
    extern __shared__ __align__(16) float smem2s[];
    __shared__ DevParams sp;
    __shared__ DirPtrs2s sd;
    __shared__ int s_dom, s_tx, s_chunk, s_begin, s_active;
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
            const int par = B.parity;
            if (threadIdx.x == 0) {
                sp = B.p;
                s_tx = B.tiles_x;
                s_chunk = B.chunk;
                s_begin = B.item_begin;
                s_active = B.steps_left > 0;
                sd.rfin = B.f[par];
                sd.rgin = B.g[par];
                sd.rfout = B.f[par ^ 1];
                sd.rgout = B.g[par ^ 1];
            }
            for (int k = threadIdx.x; k < 4 * Q2; k += blockDim.x) dir_ptrs2s(sd, B.f, B.g, par, B.p.N, k);
            cur = d;
            __syncthreads();
        }
        if (!s_active) continue;  // uniform
        const int local = item - s_begin;
        const int tile = local % s_tx;
        const int y0 = (local / s_tx) * s_chunk;
        fused2s_segment<St>(sp, sd, smem2s, tile * TX2, y0, min(y0 + s_chunk, sp.ny));
    }
}

struct Cfg2s {
    int dev = -1, per_sm = 0, sms = 0;
};

cudaError_t setup2s(const void* fn, int device, Cfg2s& cfg)
{
    if (cfg.dev == device) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem2s);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TX2, kSmem2s);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return e;
    cfg.per_sm = per_sm > 0 ? per_sm : 1;
    cfg.sms = sms;
    cfg.dev = device;
    return cudaSuccess;
}

template <class St>
struct Ops2s {
    static Cfg2s step_cfg, batch_cfg;
    static cudaError_t launch_step(lbmp_handle* h)
    {
        cudaError_t e = setup2s((const void*)step_fused2s_kernel<St>, h->device, step_cfg);
        if (e != cudaSuccess) return e;
        const int s = h->parity, d = 1 - h->parity;
        Fused2sArgs A;
        A.tiles_x = (h->grid.nx + TX2 - 1) / TX2;
        const LaunchShape L = launch_shape(h, A.tiles_x, h->grid.ny, step_cfg.per_sm, step_cfg.sms);
        A.chunk = L.chunk;
        A.nitems = L.nitems;
        DirPtrs2s D;
        for (int k = 0; k < 4 * Q2; ++k) dir_ptrs2s(D, h->f, h->g, s, h->N, k);
        D.rfin = h->f[s];
        D.rgin = h->g[s];
        D.rfout = h->f[d];
        D.rgout = h->g[d];
        step_fused2s_kernel<St><<<L.grid, TX2, kSmem2s, h->stream>>>(h->dp, A, D);
        return cudaGetLastError();
    }
    static cudaError_t prepare(int device)
    {
        return setup2s((const void*)step_batch2s_kernel<St>, device, batch_cfg);
    }
    static cudaError_t launch(const BatchDomain* table, int ndom, int nitems, int device, cudaStream_t stream)
    {
        if (batch_cfg.dev != device) return cudaErrorNotReady;  // prepare first
        if (nitems <= 0) return cudaSuccess;
        const int cap = batch_cfg.per_sm * batch_cfg.sms;
        const int grid = nitems < cap ? nitems : cap;
        step_batch2s_kernel<St><<<grid, TX2, kSmem2s, stream>>>(table, ndom, nitems);
        return cudaGetLastError();
    }
};
template <class St>
Cfg2s Ops2s<St>::step_cfg;
template <class St>
Cfg2s Ops2s<St>::batch_cfg;

}  // namespace

const Batch3Ops batch2_ops_f16 = {TX2, 1, Ops2s<StoreF16>::prepare, Ops2s<StoreF16>::launch, nullptr, 0};
const Batch3Ops batch2_ops_bf16 = {TX2, 1, Ops2s<StoreBF16>::prepare, Ops2s<StoreBF16>::launch, nullptr, 0};

cudaError_t launch_step_fused2s(lbmp_handle* h)
{
    if (h->D != 2) return cudaErrorInvalidValue;
    if (h->params.storage == LBMP_FP16_SHIFTED) return Ops2s<StoreF16>::launch_step(h);
    if (h->params.storage == LBMP_BF16_SHIFTED) return Ops2s<StoreBF16>::launch_step(h);
    return cudaErrorInvalidValue;
}

}  // namespace lbmp
