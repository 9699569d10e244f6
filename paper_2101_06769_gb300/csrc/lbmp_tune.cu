// lbmp_tune.cu -- launch-shape autotuner of the fused step kernels
// (include/lbmp.h, lbmp_autotune) and the device name query.
//
// A trial launch is the step kernel without the parity flip of lbmp_step: it
// reads the current population set and writes the other one, so the state
// the handle exposes is untouched and the next real step overwrites the
// trial's output.  The one array a step rewrites in place, the stored
// previous phi u of the reduced phase lattice, is saved before the trials
// and restored after them.
#include <stdio.h>
#include <string.h>

#include "lbmp_internal.h"

namespace lbmp {

cudaError_t phiu_save(lbmp_handle* h, cudaStream_t stream, float** copy)
{
    *copy = nullptr;
    const size_t n = phiu_bytes(h);
    if (n == 0 || !h->phiu) return cudaSuccess;
    cudaError_t e = dev_alloc(h, (void**)copy, n);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(*copy, h->phiu, n, cudaMemcpyDeviceToDevice, stream);
}

cudaError_t phiu_restore(lbmp_handle* h, cudaStream_t stream, float* copy)
{
    if (!copy) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(h->phiu, copy, phiu_bytes(h), cudaMemcpyDeviceToDevice, stream);
    const cudaError_t es = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = es;
    dev_free(h, copy, phiu_bytes(h));
    return e;
}

}  // namespace lbmp

extern "C" {

LBMP_API int lbmp_autotune(lbmp_handle* h, int reps, lbmp_tune_entry* table, int max_entries, int* n_entries)
{
    if (n_entries) *n_entries = 0;
    if (!h) return lbmp::set_error(LBMP_ERR_INVALID_ARG, "null handle");
    if (reps < 1) return lbmp::set_error(LBMP_ERR_INVALID_ARG, "reps must be >= 1");
    if (max_entries < 0) return lbmp::set_error(LBMP_ERR_INVALID_ARG, "max_entries must be >= 0");
    // nothing to tune for the reference pair; an in-place AA step cannot be
    // run as a trial (it would advance the state)
    if (h->kernel == 1 || !lbmp::fused_supported(h) || h->aa) return LBMP_OK;
    const int nmarch = h->D == 3 ? h->grid.nz : h->grid.ny;
    int chunks[10], nc = 0;
    chunks[nc++] = 0;
    for (int c = 1; c <= 128; c *= 2)  // 1 and 2 for small domains: more work items than SMs
        if (c <= nmarch) chunks[nc++] = c;
    const int ctas[4] = {0, 1, 2, 3};
    // tile shapes exist for the FP32 D3Q27 cp.async kernel only
    const int ntiles = (h->D == 3 && h->params.storage == LBMP_FP32 && h->kernel == 0 && !h->reduced) ? 3 : 1;
    const int saved_chunk = h->opt_chunk, saved_ctas = h->opt_ctas, saved_tile = h->opt_tile;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float* phiu_copy = nullptr;
    cudaError_t e = lbmp::phiu_save(h, h->stream, &phiu_copy);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best = 1e300;
    int best_chunk = saved_chunk, best_ctas = saved_ctas, best_tile = ntiles > 1 ? saved_tile : 0, n = 0;
    for (int t = 0; t < ntiles && e == cudaSuccess; ++t)
    for (int i = 0; i < nc && e == cudaSuccess; ++i)
        for (int j = 0; j < 4 && e == cudaSuccess; ++j) {
            h->opt_tile = ntiles > 1 ? t : saved_tile;
            h->opt_chunk = chunks[i];
            h->opt_ctas = ctas[j];
            e = lbmp::launch_step(h);  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = lbmp::launch_step(h);
            if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) break;
            const double per = (double)ms / reps;
            if (table && n < max_entries) table[n] = lbmp_tune_entry{chunks[i], ctas[j], per, h->opt_tile};
            ++n;
            if (per < best) {
                best = per;
                best_chunk = chunks[i];
                best_ctas = ctas[j];
                best_tile = h->opt_tile;
            }
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    const cudaError_t er = lbmp::phiu_restore(h, h->stream, phiu_copy);
    if (e == cudaSuccess) e = er;
    if (e != cudaSuccess) {
        h->opt_chunk = saved_chunk;
        h->opt_ctas = saved_ctas;
        h->opt_tile = saved_tile;
        char buf[256];
        snprintf(buf, sizeof buf, "autotune: %s", cudaGetErrorString(e));
        return lbmp::set_error(LBMP_ERR_CUDA, buf);
    }
    h->opt_chunk = best_chunk;
    h->opt_ctas = best_ctas;
    h->opt_tile = best_tile;
    if (n_entries) *n_entries = n;
    return LBMP_OK;
}

LBMP_API int lbmp_device_name(char* out, int len)
{
    if (!out || len < 1) return lbmp::set_error(LBMP_ERR_INVALID_ARG, "bad output buffer");
    int dev = 0;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, dev);
    if (e != cudaSuccess) {
        out[0] = 0;
        char buf[256];
        snprintf(buf, sizeof buf, "device name: %s", cudaGetErrorString(e));
        return lbmp::set_error(LBMP_ERR_CUDA, buf);
    }
    strncpy(out, prop.name, (size_t)len - 1);
    out[len - 1] = 0;
    return LBMP_OK;
}

}  // extern "C"
