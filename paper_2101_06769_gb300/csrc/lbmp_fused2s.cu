// lbmp_fused2s.cu -- fused single-pass D2Q9 step for the shifted 16-bit
// storage forms (and its batch form).
//
// The work decomposition of the FP32 D2Q9 kernel (lbmp_fused2.cu): a CTA owns
// a segment of TX2 cells of one row and marches through a chunk of rows; phi
// of rows y-1, y, y+1 over the segment and one side cell each way lives in
// shared memory.  A 2-D domain is at most a few MB of state, so the staging
// reads the pulled codes (2-byte loads) and the writers' references (FP32)
// straight through L1 instead of copying aligned words and reference rows:
// each thread decodes its own cell's pulled g of row y+1 (threads 0 and 1 the
// two side cells as well), sums phi from the exact parts of the values
// (phi_sum_shifted) and keeps the decoded own values for the collision.
// Decoding, the collision and the encoding are those of the reference pair
// (lbmp_kernels.cu), in the same order.
#include "lbmp_internal.h"

namespace lbmp {

namespace {

constexpr int TX2 = 128;
constexpr int Q2 = 9;
constexpr int C2 = 4;
constexpr int RW = TX2 + 2;  // row of phi incl. one side cell each way
constexpr size_t kSmem2s = sizeof(float) * (2 * Q2 * TX2) + sizeof(float2) * 4 * RW;

__device__ __forceinline__ int pmod(int v, int n)
{
    const int r = v % n;
    return r < 0 ? r + n : r;
}

// row whose phi stands for row yy: periodic wrap, or the mirrored ghost at a
// wall (reading A17)
__device__ __forceinline__ int row_src(const DevParams& p, int yy)
{
    if (yy >= 0 && yy < p.ny) return yy;
    if (p.vert_periodic) return pmod(yy, p.ny);
    return yy < 0 ? 0 : p.ny - 1;
}

// phi (hi, lo) of cell (x, row) from its pulled g; keep: the decoded values
// go to buf[a * stride]
template <class St>
__device__ __forceinline__ float2 decode_row_cell(const DevParams& p, const Pop<2, St>& g, int x, int row, bool keep,
                                                  float* buf, int stride)
{
    const long long self = (long long)row * p.nx + x;
    float hi, lo;
    phi_sum_shifted<2>(
        [&](int a, float& wr, float& wq) {
            int dir;
            const long long c = pull_src<2>(p, a, x, row, 0, self, dir);
            g.load_parts(dir, c, wr, wq);
            if (keep) buf[a * stride] = wr + wq;  // the decoded value, rounded once (= Pop::load)
        },
        hi, lo);
    return make_float2(hi, lo);
}

template <class St>
__device__ __forceinline__ void stage_row16(const DevParams& p, const Pop<2, St>& g, int tid, int x_own, int x_side,
                                            int yy, float* gbuf, float2* prow)
{
    const int row = row_src(p, yy);
    if (tid < 2) prow[tid == 0 ? 0 : RW - 1] = decode_row_cell<St>(p, g, x_side, row, false, nullptr, 0);
    prow[tid + 1] = decode_row_cell<St>(p, g, x_own, row, true, gbuf + tid, TX2);
}

// rows [y0, y1) of the segment starting at x0.  One barrier per row: the
// decoded g is private to its thread, and phi of row yy sits in slot
// (yy - y0 + 1) & 3 of four, so the row staged in an iteration is never one
// that a slower thread still reads from the previous one (a thread is at
// most one iteration ahead: it must pass that iteration's barrier first).
// Ends with a barrier, so the caller may reuse shared memory afterwards.
template <class St>
__device__ __forceinline__ void fused2s_segment(const DevParams& p, const Pop<2, St>& fin, const Pop<2, St>& gin,
                                                const Pop<2, St>& fout, const Pop<2, St>& gout, float* smem, int x0,
                                                int y0, int y1)
{
    float* gS = smem;                       // [2][9][TX2] decoded g of the staged rows
    float2* phiS = (float2*)(gS + 2 * Q2 * TX2);  // [4][RW]
    const int tid = threadIdx.x;
    const int x_own = pmod(x0 + tid, p.nx);
    const int x_side = pmod(tid == 0 ? x0 - 1 : x0 + TX2, p.nx);
    const bool valid = x0 + tid < p.nx;
    stage_row16<St>(p, gin, tid, x_own, x_side, y0 - 1, gS + Q2 * TX2, phiS);
    stage_row16<St>(p, gin, tid, x_own, x_side, y0, gS, phiS + RW);
    for (int y = y0; y < y1; ++y) {
        const int cur = (y - y0) & 1;
        const int sP = (y - y0) & 3, sC = (y - y0 + 1) & 3, sN = (y - y0 + 2) & 3;
        const long long self = (long long)y * p.nx + x_own;
        float fr[Q2];
#pragma unroll
        for (int a = 0; a < Q2; ++a) {
            int dir;
            const long long c = pull_src<2>(p, a, x_own, y, 0, self, dir);
            fr[a] = fin.load(dir, c);
        }
        stage_row16<St>(p, gin, tid, x_own, x_side, y + 1, gS + (cur ^ 1) * Q2 * TX2, phiS + sN * RW);
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
            flow_collide<2>(p, nh[C2], grad, lap, m, s, dh);
            const GFromStrided gi{gS + cur * Q2 * TX2 + tid, TX2};
            float off_f, off_g;
            rest_offsets<2, St>(p, s, dh, gi, off_f, off_g);
            collide_outputs<2>(
                p, s, DhArray{dh}, m, gi, nh[C2], nl[C2],
                EncSoA<2, St>{fout.base + self, (unsigned short*)(fout.base + p.N) + self, p.N, off_f, 0.f,
                              code_seed(p, self, 0)},
                EncSoA<2, St>{gout.base + self, (unsigned short*)(gout.base + p.N) + self, p.N, off_g, 0.f,
                              code_seed(p, self, 1)});
        }
    }
    __syncthreads();
}

struct Fused2sArgs {
    int tiles_x, chunk, nitems;
};

template <class St>
__global__ void __launch_bounds__(TX2) step_fused2s_kernel(DevParams p, Fused2sArgs A, Pop<2, St> fin,
                                                           Pop<2, St> gin, Pop<2, St> fout, Pop<2, St> gout)
{
    extern __shared__ __align__(16) float smem2s[];
    for (int item = blockIdx.x; item < A.nitems; item += gridDim.x) {
        const int tile = item % A.tiles_x;
        const int y0 = (item / A.tiles_x) * A.chunk;
        fused2s_segment<St>(p, fin, gin, fout, gout, smem2s, tile * TX2, y0, min(y0 + A.chunk, p.ny));
    }
}

template <class St>
__global__ void __launch_bounds__(TX2) step_batch2s_kernel(const BatchDomain* __restrict__ table, int ndom,
                                                           int nitems)
{
    extern __shared__ __align__(16) float smem2s[];
    __shared__ DevParams sp;
    __shared__ float* sb[4];  // f in, g in, f out, g out
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
            if (threadIdx.x == 0) {
                const BatchDomain& B = table[d];
                const int par = B.parity;
                sp = B.p;
                s_tx = B.tiles_x;
                s_chunk = B.chunk;
                s_begin = B.item_begin;
                s_active = B.steps_left > 0;
                sb[0] = B.f[par];
                sb[1] = B.g[par];
                sb[2] = B.f[par ^ 1];
                sb[3] = B.g[par ^ 1];
            }
            cur = d;
            __syncthreads();
        }
        if (!s_active) continue;  // uniform
        const int local = item - s_begin;
        const int tile = local % s_tx;
        const int y0 = (local / s_tx) * s_chunk;
        const long long N = sp.N;
        fused2s_segment<St>(sp, Pop<2, St>{sb[0], N}, Pop<2, St>{sb[1], N}, Pop<2, St>{sb[2], N},
                            Pop<2, St>{sb[3], N}, smem2s, tile * TX2, y0, min(y0 + s_chunk, sp.ny));
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
        step_fused2s_kernel<St><<<L.grid, TX2, kSmem2s, h->stream>>>(
            h->dp, A, Pop<2, St>{h->f[s], h->N}, Pop<2, St>{h->g[s], h->N}, Pop<2, St>{h->f[d], h->N},
            Pop<2, St>{h->g[d], h->N});
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

const Batch3Ops batch2_ops_f16 = {TX2, 1, Ops2s<StoreF16>::prepare, Ops2s<StoreF16>::launch};
const Batch3Ops batch2_ops_bf16 = {TX2, 1, Ops2s<StoreBF16>::prepare, Ops2s<StoreBF16>::launch};

cudaError_t launch_step_fused2s(lbmp_handle* h)
{
    if (h->D != 2) return cudaErrorInvalidValue;
    if (h->params.storage == LBMP_FP16_SHIFTED) return Ops2s<StoreF16>::launch_step(h);
    if (h->params.storage == LBMP_BF16_SHIFTED) return Ops2s<StoreBF16>::launch_step(h);
    return cudaErrorInvalidValue;
}

}  // namespace lbmp
