// lbmp_batch.cu -- batches of domains advanced by one persistent kernel per
// step (include/lbmp.h, lbmp_batch_*).
//
// The member table lives in device memory: the step kernel reads each
// member's parameters, population sets and parity from it, and a one-block
// epilogue flips the parities and counts the steps down.  Nothing a step
// needs comes from the host, so the kernels of a run of steps are captured
// once in a CUDA graph and the graph is replayed until the membership (or the
// set of members with steps left) changes.  The FP32 D3Q27 kinds run the
// member-grid form of their kernel: the members are kernel parameters with
// the population sets of the step's parity, so the graphs are captured for
// both phases (even or odd number of steps since the capture) and the batch
// replays the one of its current phase.  Members are grouped by kind --
// FP32, FP16 and BF16 (shifted storage) D3Q27, FP32 D3Q27 with the reduced
// phase lattice, then FP32, FP16 and BF16 D2Q9, FP32 D2Q9 with the reduced
// phase lattice, and FP32 D2Q9 with a symmetry x axis on either lattice --
// each kind a contiguous segment of the table with its own work numbering
// and its own persistent kernel.  Within a step the D3Q27 kernels run on the
// batch stream and the D2Q9 kernels on a forked second stream, joined before
// the epilogue.  The tile shape of the FP32 D3Q27 kernel and the planes (rows)
// per work item are options of the batch, picked by lbmp_batch_autotune.
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "lbmp_internal.h"

namespace {

constexpr int kMaxMembers = 1024;
constexpr int kGraphSteps = 16;  // steps per replay of the long graph

struct Member {
    lbmp_handle* h;
    long left;
};

// member kinds, in table order: D3Q27 kinds first, then D2Q9 kinds
enum Kind {
    kF32x3 = 0,
    kF16x3 = 1,
    kBF16x3 = 2,
    kF32x3R = 3,  // FP32 D3Q27 flow, D3Q7 phase field
    kF32x2 = 4,
    kF16x2 = 5,
    kBF16x2 = 6,
    kF32x2R = 7,   // FP32 D2Q9 flow, D2Q5 phase field
    kF32x2S = 8,   // FP32 D2Q9 with a symmetry x axis
    kF32x2RS = 9,  // the same with the D2Q5 phase field
    kKinds = 10
};
constexpr int kLast3 = kF32x3R;  // the D3Q27 kinds are kF32x3 .. kLast3

int kind_of(const lbmp_handle* h)
{
    const int st = h->params.storage;
    if (h->D == 2 && h->dp.sym_x) return h->reduced ? kF32x2RS : kF32x2S;
    if (h->D == 2 && h->reduced) return kF32x2R;
    if (h->D == 2) return st == LBMP_FP16_SHIFTED ? kF16x2 : (st == LBMP_BF16_SHIFTED ? kBF16x2 : kF32x2);
    if (h->reduced) return kF32x3R;
    return st == LBMP_FP16_SHIFTED ? kF16x3 : (st == LBMP_BF16_SHIFTED ? kBF16x3 : kF32x3);
}

}  // namespace

struct lbmp_batch {
    size_t budget;
    cudaStream_t stream;
    bool own_stream;  // created here: the legacy default stream cannot be captured
    cudaStream_t side;               // second branch of a step (D2Q9 members)
    cudaEvent_t fork, join;
    int tile, chunk;                 // D3Q27 tile shape (LBMP_OPT_TILE values), planes per item (0 = 16)
    int device;
    std::vector<Member> members;
    lbmp::BatchDomain* d_table;       // device, kMaxMembers entries, grouped by kind
    std::vector<lbmp::BatchDomain> h_table;
    int dom0[kKinds], ndom[kKinds], nitems[kKinds];  // table segment and work items per kind
    bool dirty;
    int phase;  // steps taken since the graphs were captured, mod 2
    cudaGraphExec_t g_long[2], g_one[2];
};

namespace {

// f' and g, two sets each, and the stored phi u of the reduced phase lattice
size_t state_bytes(const lbmp_handle* h)
{
    return 2 * (lbmp::set_bytes(h) + lbmp::gset_bytes(h)) + lbmp::phiu_bytes(h);
}

void drop_graphs(lbmp_batch* b)
{
    for (int k = 0; k < 2; ++k) {
        if (b->g_long[k]) cudaGraphExecDestroy(b->g_long[k]);
        if (b->g_one[k]) cudaGraphExecDestroy(b->g_one[k]);
        b->g_long[k] = b->g_one[k] = nullptr;
    }
}

int total_dom(const lbmp_batch* b)
{
    int n = 0;
    for (int k = 0; k < kKinds; ++k) n += b->ndom[k];
    return n;
}

const lbmp::Batch3Ops& ops3_of(const lbmp_batch* b, int kind)
{
    if (kind == kF16x3) return lbmp::batch3_ops_f16;
    if (kind == kBF16x3) return lbmp::batch3_ops_bf16;
    if (kind == kF32x3R) return lbmp::batch3_ops_red;
    if (kind == kF16x2) return lbmp::batch2_ops_f16;
    if (kind == kBF16x2) return lbmp::batch2_ops_bf16;
    return lbmp::batch3_ops(b->tile);
}

// the kernels of one kind of D3Q27 members: the member-grid form in groups
// of as many members as its parameters hold, else the persistent form
cudaError_t launch3(lbmp_batch* b, int kind, int flip, cudaStream_t stream)
{
    const lbmp::Batch3Ops& ops = ops3_of(b, kind);
    const int d0 = b->dom0[kind], n = b->ndom[kind];
    if (!ops.launch_grid) return ops.launch(b->d_table + d0, n, b->nitems[kind], b->device, stream);
    if (ops.grid_members <= 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < n && e == cudaSuccess; k += ops.grid_members) {
        const int m = n - k < ops.grid_members ? n - k : ops.grid_members;
        e = ops.launch_grid(b->h_table.data() + d0 + k, b->d_table + d0 + k, m, flip, b->device, stream);
    }
    return e;
}

// the step kernels of one step (no epilogue): D3Q27 kinds on the batch
// stream, D2Q9 members on the side stream when both are present; flip: the
// members' parities differ from the host table's by this step's phase
cudaError_t step_kernels(lbmp_batch* b, int flip)
{
    cudaError_t e = cudaSuccess;
    bool any3 = false;
    for (int k = kF32x3; k <= kLast3; ++k) any3 = any3 || b->ndom[k];
    bool any2 = false;
    for (int k = kF32x2; k < kKinds; ++k) any2 = any2 || b->ndom[k];
    const bool fork = any3 && any2;
    if (fork) {
        e = cudaEventRecord(b->fork, b->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->fork, 0);
    }
    for (int k = kF32x3; k <= kLast3 && e == cudaSuccess; ++k)
        if (b->ndom[k]) e = launch3(b, k, flip, b->stream);
    // FP32 D2Q9 kinds: phase lattice and x boundary as template parameters
    static const int k2[4] = {kF32x2, kF32x2R, kF32x2S, kF32x2RS};
    for (int j = 0; j < 4 && e == cudaSuccess; ++j)
        if (b->ndom[k2[j]])
            e = lbmp::launch_batch2(b->d_table + b->dom0[k2[j]], b->ndom[k2[j]], b->nitems[k2[j]], b->device,
                                    fork ? b->side : b->stream, (j & 1) != 0, j >= 2);
    for (int k = kF16x2; k <= kBF16x2 && e == cudaSuccess; ++k)
        if (b->ndom[k])
            e = ops3_of(b, k).launch(b->d_table + b->dom0[k], b->ndom[k], b->nitems[k], b->device,
                                     fork ? b->side : b->stream);
    if (e == cudaSuccess && fork) {
        e = cudaEventRecord(b->join, b->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join, 0);
    }
    return e;
}

cudaError_t capture(lbmp_batch* b, int steps, int phase, cudaGraphExec_t* out)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < steps && e == cudaSuccess; ++k) {
        e = step_kernels(b, (phase + k) & 1);
        if (e == cudaSuccess) e = lbmp::launch_batch_epilogue(b->d_table, total_dom(b), b->stream);
    }
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

// Rebuild the device table from the members with steps left (grouped by
// kind, each kind with its own work numbering), and (graphs) the graphs.
cudaError_t rebuild(lbmp_batch* b, bool graphs = true)
{
    drop_graphs(b);
    b->h_table.clear();
    for (int kind = 0; kind < kKinds; ++kind) {
    b->dom0[kind] = (int)b->h_table.size();
    const int D = kind >= kF32x2 ? 2 : 3;
    int item = 0;
    const bool fp32_2d = kind == kF32x2 || kind == kF32x2R || kind == kF32x2S || kind == kF32x2RS;
    const int TX = fp32_2d ? lbmp::batch2_tile_x() : ops3_of(b, kind).tile_x;
    const int TY = D == 3 ? ops3_of(b, kind).tile_y : 1;
    const int chunk = b->chunk > 0 ? b->chunk : 16;
    for (const Member& m : b->members) {
        if (m.left <= 0 || kind_of(m.h) != kind) continue;
        const lbmp_handle* h = m.h;
        lbmp::BatchDomain d;
        memset(&d, 0, sizeof d);
        d.p = h->dp;
        d.p.step = (unsigned)h->step;
        d.f[0] = h->f[0];
        d.f[1] = h->f[1];
        d.g[0] = h->g[0];
        d.g[1] = h->g[1];
        d.phiu = h->phiu;
        d.parity = h->parity;
        d.steps_left = (int)(m.left < (1L << 30) ? m.left : (1L << 30));
        // the march axis: z in 3-D, y in 2-D (one row of TX cells per tile)
        const int nmarch = D == 3 ? h->grid.nz : h->grid.ny;
        d.tiles_x = (h->grid.nx + TX - 1) / TX;
        d.tiles_y = D == 3 ? (h->grid.ny + TY - 1) / TY : 1;
        d.chunk = nmarch < chunk ? nmarch : chunk;
        d.item_begin = item;
        d.items = d.tiles_x * d.tiles_y * ((nmarch + d.chunk - 1) / d.chunk);
        item += d.items;
        b->h_table.push_back(d);
    }
    b->ndom[kind] = (int)b->h_table.size() - b->dom0[kind];
    b->nitems[kind] = item;
    }
    const int ndom = total_dom(b);
    cudaError_t e = cudaSuccess;
    if (ndom > 0) {
        for (int k = kF32x3; k <= kLast3 && e == cudaSuccess; ++k)
            if (b->ndom[k]) e = ops3_of(b, k).prepare(b->device);
        if (e == cudaSuccess && b->ndom[kF32x2]) e = lbmp::prepare_batch2(b->device, false, false);
        if (e == cudaSuccess && b->ndom[kF32x2R]) e = lbmp::prepare_batch2(b->device, true, false);
        if (e == cudaSuccess && b->ndom[kF32x2S]) e = lbmp::prepare_batch2(b->device, false, true);
        if (e == cudaSuccess && b->ndom[kF32x2RS]) e = lbmp::prepare_batch2(b->device, true, true);
        for (int k = kF16x2; k <= kBF16x2 && e == cudaSuccess; ++k)
            if (b->ndom[k]) e = ops3_of(b, k).prepare(b->device);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_table, b->h_table.data(), sizeof(lbmp::BatchDomain) * ndom,
                                cudaMemcpyHostToDevice, b->stream);
        for (int ph = 0; ph < 2 && e == cudaSuccess && graphs; ++ph) {
            e = capture(b, kGraphSteps, ph, &b->g_long[ph]);
            if (e == cudaSuccess) e = capture(b, 1, ph, &b->g_one[ph]);
        }
    }
    b->phase = 0;  // the host table holds the members' current parities
    if (e == cudaSuccess) b->dirty = !graphs;
    return e;
}

int batch_fail(int code, const char* msg) { return lbmp::set_error(code, msg); }

int batch_cuda_fail(cudaError_t e, const char* where)
{
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    return lbmp::set_error(LBMP_ERR_CUDA, buf);
}

}  // namespace

extern "C" {

LBMP_API int lbmp_batch_create(size_t hbm_budget, void* cuda_stream, lbmp_batch** out)
{
    if (!out) return batch_fail(LBMP_ERR_INVALID_ARG, "null output");
    *out = nullptr;
    lbmp_batch* b = new (std::nothrow) lbmp_batch();
    if (!b) return batch_fail(LBMP_ERR_NOMEM, "host allocation failed");
    b->budget = hbm_budget;
    b->stream = (cudaStream_t)cuda_stream;
    b->own_stream = false;
    b->side = nullptr;
    b->fork = b->join = nullptr;
    b->tile = 0;
    b->chunk = 0;
    b->d_table = nullptr;
    for (int k = 0; k < kKinds; ++k) b->dom0[k] = b->ndom[k] = b->nitems[k] = 0;
    b->dirty = true;
    b->phase = 0;
    b->g_long[0] = b->g_long[1] = b->g_one[0] = b->g_one[1] = nullptr;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess && !b->stream) {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_table, sizeof(lbmp::BatchDomain) * kMaxMembers);
    if (e != cudaSuccess) {
        if (b->fork) cudaEventDestroy(b->fork);
        if (b->join) cudaEventDestroy(b->join);
        if (b->side) cudaStreamDestroy(b->side);
        if (b->own_stream) cudaStreamDestroy(b->stream);
        delete b;
        return batch_cuda_fail(e, "batch table");
    }
    *out = b;
    return LBMP_OK;
}

LBMP_API int lbmp_batch_destroy(lbmp_batch* b)
{
    if (!b) return LBMP_OK;
    cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    if (b->d_table) cudaFree(b->d_table);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return LBMP_OK;
}

LBMP_API int lbmp_batch_add(lbmp_batch* b, lbmp_handle* h, long steps)
{
    if (!b || !h) return batch_fail(LBMP_ERR_INVALID_ARG, "null argument");
    if (steps <= 0) return batch_fail(LBMP_ERR_INVALID_ARG, "steps must be > 0");
    if (h->device != b->device) return batch_fail(LBMP_ERR_INVALID_ARG, "domain lives on another device");
    if ((int)b->members.size() >= kMaxMembers) return batch_fail(LBMP_ERR_INVALID_ARG, "batch is full");
    if (h->divu) return batch_fail(LBMP_ERR_UNSUPPORTED, "divergence-term domains are not batch members");
    if (h->slab || h->aa) return batch_fail(LBMP_ERR_UNSUPPORTED, "z-slabs and in-place AA domains are not batch members");
    size_t used = 0;
    for (const Member& m : b->members) {
        if (m.h == h) return batch_fail(LBMP_ERR_INVALID_ARG, "domain is already a member");
        used += state_bytes(m.h);
    }
    if (b->budget && used + state_bytes(h) > b->budget)
        return batch_fail(LBMP_ERR_NOMEM, "domain does not fit the batch's HBM budget");
    // the member's own stream may still have work queued: order it before the batch's
    if (h->stream != b->stream) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return batch_cuda_fail(e, "member stream");
    }
    b->members.push_back(Member{h, steps});
    b->dirty = true;
    return LBMP_OK;
}

LBMP_API int lbmp_batch_remove(lbmp_batch* b, lbmp_handle* h)
{
    if (!b || !h) return batch_fail(LBMP_ERR_INVALID_ARG, "null argument");
    for (size_t k = 0; k < b->members.size(); ++k)
        if (b->members[k].h == h) {
            cudaError_t e = cudaStreamSynchronize(b->stream);
            if (e != cudaSuccess) return batch_cuda_fail(e, "batch stream");
            b->members.erase(b->members.begin() + (long)k);
            b->dirty = true;
            return LBMP_OK;
        }
    return batch_fail(LBMP_ERR_INVALID_ARG, "domain is not a member");
}

LBMP_API int lbmp_batch_step(lbmp_batch* b, long n, int* n_finished)
{
    if (!b) return batch_fail(LBMP_ERR_INVALID_ARG, "null batch");
    if (n < 0) return batch_fail(LBMP_ERR_INVALID_ARG, "negative step count");
    if (n_finished) *n_finished = 0;
    cudaError_t e = cudaSuccess;
    if (b->dirty) e = rebuild(b);
    if (e != cudaSuccess) return batch_cuda_fail(e, "batch rebuild");
    const int ndom = total_dom(b);
    if (ndom == 0 || n == 0) return LBMP_OK;
    // never run more steps than the longest member still needs
    long need = 0;
    for (const Member& m : b->members) need = m.left > need ? m.left : need;
    if (n > need) n = need;
    // a long graph takes an even number of steps: the phase stays
    for (long k = 0; k + kGraphSteps <= n && e == cudaSuccess; k += kGraphSteps)
        e = cudaGraphLaunch(b->g_long[b->phase], b->stream);
    for (long k = 0; k < n % kGraphSteps && e == cudaSuccess; ++k) {
        e = cudaGraphLaunch(b->g_one[b->phase], b->stream);
        b->phase ^= 1;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->h_table.data(), b->d_table, sizeof(lbmp::BatchDomain) * ndom, cudaMemcpyDeviceToHost,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_cuda_fail(e, "batch step");
    // write the device bookkeeping back to the member handles (table order:
    // kinds in order, each in membership order)
    int finished = 0, t = 0;
    for (int kind = 0; kind < kKinds; ++kind)
    for (Member& m : b->members) {
        if (m.left <= 0 || kind_of(m.h) != kind) continue;
        const lbmp::BatchDomain& d = b->h_table[t++];
        const long done = m.left - d.steps_left;
        m.h->parity = d.parity;
        m.h->step += done;
        m.left = d.steps_left;
        if (m.left == 0) {
            ++finished;
            b->dirty = true;  // its work leaves the table at the next step
        }
    }
    if (n_finished) *n_finished = finished;
    return LBMP_OK;
}

LBMP_API int lbmp_batch_autotune(lbmp_batch* b, int reps, lbmp_tune_entry* table, int max_entries, int* n_entries)
{
    if (n_entries) *n_entries = 0;
    if (!b) return batch_fail(LBMP_ERR_INVALID_ARG, "null batch");
    if (reps < 1) return batch_fail(LBMP_ERR_INVALID_ARG, "reps must be >= 1");
    if (max_entries < 0) return batch_fail(LBMP_ERR_INVALID_ARG, "max_entries must be >= 0");
    const int saved_tile = b->tile, saved_chunk = b->chunk;
    const int chunks[4] = {8, 16, 32, 64};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    // the trials run real step kernels: keep the reduced members' stored phi u
    std::vector<float*> phiu_copies(b->members.size(), nullptr);
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < b->members.size() && e == cudaSuccess; ++k)
        e = lbmp::phiu_save(b->members[k].h, b->stream, &phiu_copies[k]);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // two passes over the shapes, each shape's time the smaller of its two
    // trials: one slow or fast trial (a clock change, another process) does
    // not decide the pick
    double per_shape[3][4];
    for (int t = 0; t < 3; ++t)
        for (int i = 0; i < 4; ++i) per_shape[t][i] = 1e300;
    bool any = false;
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass)
        for (int t = 0; t < 3 && e == cudaSuccess; ++t)
            for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
                b->tile = t;
                b->chunk = chunks[i];
                e = rebuild(b, false);  // table only; trial launches have no epilogue
                if (e != cudaSuccess || total_dom(b) == 0) break;
                e = step_kernels(b, 0);  // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
                for (int r = 0; r < reps && e == cudaSuccess; ++r) e = step_kernels(b, 0);
                if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) break;
                const double per = (double)ms / reps;
                if (per < per_shape[t][i]) per_shape[t][i] = per;
                any = true;
            }
    double best = 1e300;
    int best_tile = saved_tile, best_chunk = saved_chunk, n = 0;
    for (int t = 0; t < 3 && any; ++t)
        for (int i = 0; i < 4; ++i) {
            const double per = per_shape[t][i];
            if (per >= 1e300) continue;
            if (table && n < max_entries) table[n] = lbmp_tune_entry{chunks[i], 0, per, t};
            ++n;
            if (per < best) {
                best = per;
                best_tile = t;
                best_chunk = chunks[i];
            }
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    // the D2Q9 trials ran on the side stream, joined into b->stream
    for (size_t k = 0; k < b->members.size(); ++k) {
        const cudaError_t er = lbmp::phiu_restore(b->members[k].h, b->stream, phiu_copies[k]);
        if (e == cudaSuccess) e = er;
    }
    b->tile = n ? best_tile : saved_tile;
    b->chunk = n ? best_chunk : saved_chunk;
    b->dirty = true;  // graphs are rebuilt with the chosen shape at the next step
    if (e != cudaSuccess) return batch_cuda_fail(e, "batch autotune");
    if (n_entries) *n_entries = n;
    return LBMP_OK;
}

LBMP_API int lbmp_batch_members(const lbmp_batch* b, lbmp_handle** members, long* steps_left, int max)
{
    if (!b) return batch_fail(LBMP_ERR_INVALID_ARG, "null batch");
    const int n = (int)b->members.size();
    for (int k = 0; k < n && k < max; ++k) {
        if (members) members[k] = b->members[k].h;
        if (steps_left) steps_left[k] = b->members[k].left;
    }
    return n;
}

}  // extern "C"
