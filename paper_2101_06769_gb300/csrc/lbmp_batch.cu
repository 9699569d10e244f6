// lbmp_batch.cu -- batches of domains advanced by one persistent kernel per
// step (include/lbmp.h, lbmp_batch_*).
//
// The member table lives in device memory: the step kernel reads each
// member's parameters, population sets and parity from it, and a one-block
// epilogue flips the parities and counts the steps down.  Nothing a step
// needs comes from the host, so the kernels of a run of steps are captured
// once in a CUDA graph and the graph is replayed until the membership (or the
// set of members with steps left) changes.  Within a step the D3Q27 and the
// D2Q9 batch kernels run on two forked streams (independent members), joined
// before the epilogue.  The tile shape of the D3Q27 kernel and the planes
// (rows) per work item are options of the batch, picked by
// lbmp_batch_autotune.
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
    lbmp::BatchDomain* d_table;       // device, kMaxMembers entries: 3-D members, then 2-D members
    std::vector<lbmp::BatchDomain> h_table;
    int ndom3, nitems3, ndom2, nitems2;
    bool dirty;
    cudaGraphExec_t g_long, g_one;
};

namespace {

size_t state_bytes(const lbmp_handle* h) { return 2 * lbmp::set_bytes(h) * 2; }  // f' and g, two sets each

void drop_graphs(lbmp_batch* b)
{
    if (b->g_long) cudaGraphExecDestroy(b->g_long);
    if (b->g_one) cudaGraphExecDestroy(b->g_one);
    b->g_long = b->g_one = nullptr;
}

// the step kernels of one step (no epilogue): D3Q27 members on the batch
// stream, D2Q9 members on the side stream when both kinds are present
cudaError_t step_kernels(lbmp_batch* b)
{
    cudaError_t e = cudaSuccess;
    const bool fork = b->ndom3 && b->ndom2;
    if (fork) {
        e = cudaEventRecord(b->fork, b->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->fork, 0);
    }
    if (e == cudaSuccess && b->ndom3)
        e = lbmp::batch3_ops(b->tile).launch(b->d_table, b->ndom3, b->nitems3, b->device, b->stream);
    if (e == cudaSuccess && b->ndom2)
        e = lbmp::launch_batch2(b->d_table + b->ndom3, b->ndom2, b->nitems2, b->device, fork ? b->side : b->stream);
    if (e == cudaSuccess && fork) {
        e = cudaEventRecord(b->join, b->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join, 0);
    }
    return e;
}

cudaError_t capture(lbmp_batch* b, int steps, cudaGraphExec_t* out)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    for (int k = 0; k < steps && e == cudaSuccess; ++k) {
        e = step_kernels(b);
        if (e == cudaSuccess) e = lbmp::launch_batch_epilogue(b->d_table, b->ndom3 + b->ndom2, b->stream);
    }
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

// Rebuild the device table from the members with steps left (3-D members
// first, then 2-D, each with its own work numbering), and (graphs) the graphs.
cudaError_t rebuild(lbmp_batch* b, bool graphs = true)
{
    drop_graphs(b);
    b->h_table.clear();
    b->ndom3 = b->nitems3 = b->ndom2 = b->nitems2 = 0;
    for (int D = 3; D >= 2; --D) {
    int item = 0;
    const lbmp::Batch3Ops& ops3 = lbmp::batch3_ops(b->tile);
    const int TX = D == 3 ? ops3.tile_x : lbmp::batch2_tile_x(), TY = D == 3 ? ops3.tile_y : 1;
    const int chunk = b->chunk > 0 ? b->chunk : 16;
    for (const Member& m : b->members) {
        if (m.left <= 0 || m.h->D != D) continue;
        const lbmp_handle* h = m.h;
        lbmp::BatchDomain d;
        memset(&d, 0, sizeof d);
        d.p = h->dp;
        d.f[0] = h->f[0];
        d.f[1] = h->f[1];
        d.g[0] = h->g[0];
        d.g[1] = h->g[1];
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
    if (D == 3) {
        b->ndom3 = (int)b->h_table.size();
        b->nitems3 = item;
    } else {
        b->ndom2 = (int)b->h_table.size() - b->ndom3;
        b->nitems2 = item;
    }
    }
    const int ndom = b->ndom3 + b->ndom2;
    cudaError_t e = cudaSuccess;
    if (ndom > 0) {
        if (b->ndom3) e = lbmp::batch3_ops(b->tile).prepare(b->device);
        if (e == cudaSuccess && b->ndom2) e = lbmp::prepare_batch2(b->device);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_table, b->h_table.data(), sizeof(lbmp::BatchDomain) * ndom,
                                cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess && graphs) e = capture(b, kGraphSteps, &b->g_long);
        if (e == cudaSuccess && graphs) e = capture(b, 1, &b->g_one);
    }
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
    b->ndom3 = b->nitems3 = b->ndom2 = b->nitems2 = 0;
    b->dirty = true;
    b->g_long = b->g_one = nullptr;
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
    if (h->params.storage != LBMP_FP32)
        return batch_fail(LBMP_ERR_UNSUPPORTED, "batch members must use FP32 storage");
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
    const int ndom = b->ndom3 + b->ndom2;
    if (ndom == 0 || n == 0) return LBMP_OK;
    // never run more steps than the longest member still needs
    long need = 0;
    for (const Member& m : b->members) need = m.left > need ? m.left : need;
    if (n > need) n = need;
    for (long k = 0; k + kGraphSteps <= n && e == cudaSuccess; k += kGraphSteps) e = cudaGraphLaunch(b->g_long, b->stream);
    for (long k = 0; k < n % kGraphSteps && e == cudaSuccess; ++k) e = cudaGraphLaunch(b->g_one, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->h_table.data(), b->d_table, sizeof(lbmp::BatchDomain) * ndom, cudaMemcpyDeviceToHost,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_cuda_fail(e, "batch step");
    // write the device bookkeeping back to the member handles (table order:
    // 3-D members, then 2-D members, each in membership order)
    int finished = 0, t = 0;
    for (int D = 3; D >= 2; --D)
    for (Member& m : b->members) {
        if (m.left <= 0 || m.h->D != D) continue;
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
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 1e300;
    int best_tile = saved_tile, best_chunk = saved_chunk, n = 0;
    for (int t = 0; t < 3 && e == cudaSuccess; ++t)
        for (int i = 0; i < 4 && e == cudaSuccess; ++i) {
            b->tile = t;
            b->chunk = chunks[i];
            e = rebuild(b, false);  // table only; trial launches have no epilogue
            if (e != cudaSuccess || b->ndom3 + b->ndom2 == 0) break;
            e = step_kernels(b);  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = step_kernels(b);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) break;
            const double per = (double)ms / reps;
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
