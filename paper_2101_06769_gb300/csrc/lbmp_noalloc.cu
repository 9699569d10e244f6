// lbmp_noalloc.cu -- lbmp_mass_noalloc: the FP64 mass reduction of the
// observables, for callers that cannot allocate device memory.
//
// Who cannot allocate: code that runs where cudaMalloc is unavailable or not
// allowed. Examples are a host framework that owns every byte of device memory
// and hands out only views into its own pool, a real-time loop with a fixed
// memory budget, or a plug-in that may not create allocations behind its
// host's back. Such a caller owns the population arrays and can still ask for
// the conserved mass, but it cannot provide (and must not trigger) a scratch
// allocation.
//
// The two-pass block reduction of lbmp_observables keeps its per-block
// partial sums in memory allocated at lbmp_create. Here the partial sums live
// in a file-scope device array of fixed size instead, so a call allocates
// nothing: no cudaMalloc, no cudaFree, no allocating library routine.
//
// Limits and sharing:
//   * one partial sum per chunk of kChunk = 2^21 values, at most kMaxPartials =
//     4096 partials (32 KiB per GPU, resident on every GPU that loads the
//     library until the process exits), hence at most 2^33 values per call;
//     larger requests are rejected with LBMP_ERR_INVALID_ARG;
//   * every call on a device shares the array, which keeps the last call's
//     contents. Nothing needs clearing: the first kernel writes every partial
//     that the second kernel reads. Calls that overlap on the GPU (on
//     different streams, or from several host threads) race on the array and
//     must be serialised by the caller;
//   * the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress, with that device current. Make that first call
//     before any stream capture. Every later call made outside a stream
//     capture looks the address up again, because a device reset
//     (cudaDeviceReset) reloads the module and moves the array; a call made
//     while its stream is capturing uses the address found by the last call
//     on that device that was not.
#include <atomic>

#include "lbmp_internal.h"

namespace {

constexpr long long kChunk = 1LL << 21;
constexpr int kMaxPartials = 4096;
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

// [0, kMaxPartials): per-chunk partial sums; [kMaxPartials]: the result
static __device__ __align__(256) double g_mass_scratch[kMaxPartials + 1];

// device address of g_mass_scratch per device ordinal (host side)
std::atomic<double*> g_scratch_addr[kMaxDevices];

__global__ void __launch_bounds__(kThreads) mass_partial_kernel(const float* __restrict__ v, long long n,
                                                                double* __restrict__ part)
{
    __shared__ double sm[kThreads];
    const long long begin = (long long)blockIdx.x * kChunk;
    const long long end = min(begin + kChunk, n);
    double s = 0.0;
    for (long long i = begin + threadIdx.x; i < end; i += kThreads) s += (double)v[i];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void __launch_bounds__(kThreads) mass_final_kernel(const double* __restrict__ part, int nparts,
                                                              double* __restrict__ result)
{
    __shared__ double sm[kThreads];
    double s = 0.0;
    for (int b = threadIdx.x; b < nparts; b += kThreads) s += part[b];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *result = sm[0];
}

int noalloc_fail(int code, const char* msg) { return lbmp::set_error(code, msg); }

}  // namespace

extern "C" {

LBMP_API int lbmp_mass_noalloc(const float* g_dev, long long n_values, double* mass_out, void* cuda_stream)
{
    if (!g_dev || !mass_out) return noalloc_fail(LBMP_ERR_INVALID_ARG, "lbmp_mass_noalloc: null pointer");
    if (n_values < 0) return noalloc_fail(LBMP_ERR_INVALID_ARG, "lbmp_mass_noalloc: negative size");
    const long long nparts = (n_values + kChunk - 1) / kChunk;
    if (nparts > kMaxPartials)
        return noalloc_fail(LBMP_ERR_INVALID_ARG,
                            "lbmp_mass_noalloc: more than 2^33 values (the fixed scratch holds 4096 partial "
                            "sums of 2^21 values each)");
    if (n_values == 0) {
        *mass_out = 0.0;
        return LBMP_OK;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(LBMP_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(LBMP_ERR_UNSUPPORTED, "lbmp_mass_noalloc: device ordinal");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return noalloc_fail(LBMP_ERR_CUDA, cudaGetErrorString(e));
    double* scratch = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (cap == cudaStreamCaptureStatusNone) {
        // set-up with this device current: on the first call, and again on
        // every call outside a capture (a device reset moves the array)
        double* fresh = nullptr;
        e = cudaGetSymbolAddress((void**)&fresh, g_mass_scratch);
        if (e != cudaSuccess || !fresh) {
            return noalloc_fail(LBMP_ERR_CUDA, e != cudaSuccess ? cudaGetErrorString(e)
                                                                : "lbmp_mass_noalloc: null symbol address");
        }
        scratch = fresh;
        g_scratch_addr[dev].store(scratch, std::memory_order_release);
    } else if (!scratch) {
        return noalloc_fail(LBMP_ERR_UNSUPPORTED,
                            "lbmp_mass_noalloc: first call on this device made during a stream capture "
                            "(make one call before capturing)");
    }
    // an earlier, unrelated launch error is not this call's: clear it first
    (void)cudaGetLastError();
    mass_partial_kernel<<<(unsigned)nparts, kThreads, 0, s>>>(g_dev, n_values, scratch);
    mass_final_kernel<<<1, kThreads, 0, s>>>(scratch, (int)nparts, scratch + kMaxPartials);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(mass_out, scratch + kMaxPartials, sizeof(double),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return noalloc_fail(LBMP_ERR_CUDA, cudaGetErrorString(e));
    return LBMP_OK;
}

}  // extern "C"
