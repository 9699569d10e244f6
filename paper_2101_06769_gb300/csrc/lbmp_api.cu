// lbmp_api.cu -- extern "C" entry points of the library (include/lbmp.h):
// argument validation, the parameter closure of the paper's problem statement,
// device allocation, state transfer and error reporting.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include <limits>

#include "lbmp_internal.h"

namespace {

thread_local char g_msg[512] = "";

int fail(int code, const char* fmt, const char* detail = nullptr)
{
    if (detail)
        snprintf(g_msg, sizeof g_msg, fmt, detail);
    else
        snprintf(g_msg, sizeof g_msg, "%s", fmt);
    return code;
}

int cuda_fail(cudaError_t e, const char* where)
{
    snprintf(g_msg, sizeof g_msg, "%s: %s", where, cudaGetErrorString(e));
    return LBMP_ERR_CUDA;
}

#define LBMP_CUDA(call, where)                         \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

// Problem statement -> lattice parameters (Sec. 2.1, 2.2, 3):
//   rho_h = 1; rho_l = 1/ratio or (1-At)/(1+At);
//   U = U0, or sqrt(g L) for gravity-driven cases; nu_h = U L / Re;
//   sigma = rho_h L U^2 / We (rho_l with LBMP_FLAG_WE_LIGHT);
//   beta = 12 sigma/W, kappa = 3 sigma W/2; tau_phi = M/cs2 + 1/2 with the
//   phase lattice's cs2 (1/4 on D3Q7, else 1/3), lambda_phi = 1 - 1/(2 tau_phi).
int derive(const lbmp_params& p, int D, lbmp_derived& d)
{
    memset(&d, 0, sizeof d);
    d.rho_h = 1.0;
    if (p.atwood > 0.0) {
        if (!(p.atwood < 1.0)) return fail(LBMP_ERR_INVALID_ARG, "atwood must lie in (0, 1)");
        d.rho_l = (1.0 - p.atwood) / (1.0 + p.atwood);
    } else {
        if (!(p.rho_ratio > 0.0)) return fail(LBMP_ERR_INVALID_ARG, "rho_ratio must be > 0");
        d.rho_l = 1.0 / p.rho_ratio;
    }
    d.U_ref = (p.U0 > 0.0) ? p.U0 : sqrt(p.g_accel > 0.0 ? p.g_accel * p.L_ref : 0.0);
    if (p.nu_h > 0.0) {
        d.nu_h = p.nu_h;
    } else {
        if (!(p.Re > 0.0 && p.L_ref > 0.0 && d.U_ref > 0.0))
            return fail(LBMP_ERR_INVALID_ARG, "viscosity: give nu_h > 0, or Re, L_ref and U0 or g_accel");
        d.nu_h = d.U_ref * p.L_ref / p.Re;
    }
    if (!(p.nu_ratio > 0.0)) return fail(LBMP_ERR_INVALID_ARG, "nu_ratio must be > 0");
    d.nu_l = d.nu_h * p.nu_ratio;
    if (p.sigma >= 0.0)
        d.sigma = p.sigma;
    else if (p.We > 0.0)
        d.sigma = ((p.flags & LBMP_FLAG_WE_LIGHT) ? d.rho_l : d.rho_h) * p.L_ref * d.U_ref * d.U_ref / p.We;
    else
        d.sigma = 0.0;
    if (!(p.width > 0.0)) return fail(LBMP_ERR_INVALID_ARG, "width W must be > 0");
    if (!(p.mobility > 0.0)) return fail(LBMP_ERR_INVALID_ARG, "mobility M must be > 0");
    d.W = p.width;
    d.M = p.mobility;
    d.beta = 12.0 * d.sigma / d.W;
    d.kappa = 1.5 * d.sigma * d.W;
    const double cs2g = ((p.flags & LBMP_FLAG_PHASE_REDUCED) && D == 3) ? 0.25 : 1.0 / 3.0;
    d.tau_phi = d.M / cs2g + 0.5;
    d.lambda_phi = 1.0 - 0.5 / d.tau_phi;
    d.g_accel = p.g_accel;
    d.force_x = p.force_x;
    if (!isfinite(d.nu_h) || !isfinite(d.nu_l) || !isfinite(d.sigma))
        return fail(LBMP_ERR_INVALID_ARG, "non-finite derived parameter");
    return LBMP_OK;
}

void fill_devparams(lbmp_handle* h)
{
    lbmp::DevParams& q = h->dp;
    const lbmp_derived& d = h->der;
    q.nx = h->grid.nx;
    q.ny = h->grid.ny;
    q.nz = h->grid.nz;
    q.vert_periodic = h->grid.periodic[h->D - 1] ? 1 : 0;
    q.sym_x = (h->D == 2 && h->grid.periodic[0] == 2) ? 1 : 0;
    // a plain domain; lbmp_create_slab overrides these for one rank's slab
    q.wall_lo = q.wall_hi = q.vert_periodic ? 0 : 1;
    q.zb = 0;
    q.ze = h->D == 3 ? h->grid.nz : h->grid.ny;
    q.zoff = 0;
    q.nzg = q.ze;
    q.aa = 0;  // lbmp_create sets the phase of an AA domain
    q.N = h->N;
    q.rho_l = (float)d.rho_l;
    q.drho = (float)(d.rho_h - d.rho_l);
    q.rho_bar = (float)(0.5 * (d.rho_h + d.rho_l));
    q.nu_h = (float)d.nu_h;
    q.nu_l = (float)d.nu_l;
    q.eta_h = (float)(d.rho_h * d.nu_h);
    q.eta_l = (float)(d.rho_l * d.nu_l);
    q.beta2 = (float)(2.0 * d.beta);
    q.kappa = (float)d.kappa;
    q.inv_tau_phi = (float)(1.0 / d.tau_phi);
    q.lam_sharp = (float)(d.lambda_phi * 4.0 / d.W);
    q.lam_corr = (float)(d.lambda_phi * ((h->reduced && h->D == 3) ? 4.0 : 3.0));
    q.g_accel = (float)d.g_accel;
    q.force_x = (float)d.force_x;
    q.flags = h->params.flags;
    q.wait_ns = 2000000000ull;  // 2 s
    q.test_extra_tx = 0;
}

void drop_step_graphs(lbmp_handle* h)
{
    for (int k = 0; k < 2; ++k)
        if (h->step_graph[k]) {
            cudaGraphExecDestroy(h->step_graph[k]);
            h->step_graph[k] = nullptr;
        }
    h->graph_warm = false;
}

// bytes of the observables' result slots: 16 scalars and phi on the spike and bubble columns
size_t red_out_bytes(const lbmp_handle* h)
{
    const int nv = (h->D == 3) ? h->grid.nz : h->grid.ny;
    return sizeof(double) * (16 + 2 * (size_t)nv);
}

void free_handle(lbmp_handle* h)
{
    drop_step_graphs(h);
    for (int k = 0; k < 2; ++k) {
        if (k == 1 && h->aa) break;  // f[1], g[1] alias the single AA set
        lbmp::dev_free(h, h->f[k], lbmp::set_bytes(h));
        lbmp::dev_free(h, h->g[k], lbmp::gset_bytes(h));
    }
    lbmp::dev_free(h, h->phi, 2 * sizeof(float) * (size_t)h->N);
    lbmp::dev_free(h, h->phiu, lbmp::phiu_bytes(h));
    for (int k = 0; k < 2; ++k) lbmp::dev_free(h, h->uvel[k], lbmp::uvel_bytes(h));
    lbmp::dev_free(h, h->red, sizeof(double) * 4 * (size_t)h->red_blocks);
    lbmp::dev_free(h, h->red_out, red_out_bytes(h));
    delete h;
}

// observables: a speed above this marks the run unstable (health bit 1)
constexpr double kMaxSpeed = 0.35;

// slot of red_out (a double) that holds the device status word (an int);
// slots 0-5 take the observables, 12-15 the reference mass, 16- the columns
constexpr int kStatusSlot = 8;

// LBMP_ERR_TIMEOUT if a step kernel recorded a bounded wait that ran out
int status_of(int word)
{
    if (word & lbmp::kStatusWaitTimeout)
        return fail(LBMP_ERR_TIMEOUT, "a bounded wait of a step kernel ran out; the state is invalid");
    return LBMP_OK;
}

int check_handle(const lbmp_handle* h)
{
    if (!h) return fail(LBMP_ERR_INVALID_ARG, "null handle");
    return LBMP_OK;
}

}  // namespace

namespace lbmp {
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }

cudaError_t dev_alloc(lbmp_handle* h, void** p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    if (!h->alloc.alloc) return cudaMalloc(p, bytes);
    *p = h->alloc.alloc(bytes, (void*)h->stream, h->alloc.ctx);
    if (!*p) return cudaErrorMemoryAllocation;
    if (((uintptr_t)*p) & 255u) {  // the kernels' vector and bulk accesses need the promised alignment
        h->alloc.free(*p, bytes, (void*)h->stream, h->alloc.ctx);
        *p = nullptr;
        return cudaErrorMisalignedAddress;
    }
    return cudaSuccess;
}

void dev_free(lbmp_handle* h, void* p, size_t bytes)
{
    if (!p) return;
    if (h->alloc.free)
        h->alloc.free(p, bytes, (void*)h->stream, h->alloc.ctx);
    else
        cudaFree(p);
}

cudaError_t ensure_phi(lbmp_handle* h)
{
    if (h->phi) return cudaSuccess;
    return dev_alloc(h, (void**)&h->phi, 2 * sizeof(float) * (size_t)h->N);
}

cudaError_t launch_step(lbmp_handle* h)
{
    if (h->aa) return launch_step_aa(h);
    if (h->kernel == 1 || !fused_supported(h)) return launch_step_simple(h);
    if (h->params.storage != LBMP_FP32) return h->D == 3 ? launch_step_fused16(h) : launch_step_fused2s(h);
    if (h->D == 2) return launch_step_fused2(h);
    if (h->reduced) return launch_step_fused3_red(h);
    if (h->kernel == 2 && bulk_supported(h)) return launch_step_fused_bulk(h);
    if (h->opt_tile == 1) return launch_step_fused3_t16x8(h);
    if (h->opt_tile == 2) return launch_step_fused3_t8x16(h);
    return launch_step_fused3(h);
}
}  // namespace lbmp

namespace {

// Runs of kStepGraph steps are replayed from a CUDA graph captured once per
// starting parity: for a small domain the host launch cost exceeds the
// kernel's own time.  kStepGraph is even, so a replay returns to the parity
// it started from.  Only for FP32 storage (the shifted forms seed their
// stochastic rounding with the step index, which a replay cannot advance),
// on a stream of the caller's (the legacy default stream cannot be
// captured) that is not itself being captured.
constexpr int kStepGraph = 16;

bool step_graph_usable(lbmp_handle* h)
{
    if (h->graph_off || h->params.storage != LBMP_FP32 || !h->stream) return false;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return st == cudaStreamCaptureStatusNone;
}

// drop the graphs when a launch option they were captured with has changed
void check_graph_key(lbmp_handle* h)
{
    const long long key[6] = {h->kernel, h->opt_chunk, h->opt_ctas, h->opt_tile, (long long)h->dp.wait_ns,
                              (long long)h->dp.test_extra_tx};
    if (memcmp(key, h->graph_key, sizeof key) != 0) {
        drop_step_graphs(h);
        memcpy(h->graph_key, key, sizeof key);
    }
}

// the graph of kStepGraph steps from the current parity (built on first use),
// or null when capture is not possible
cudaGraphExec_t step_graph(lbmp_handle* h)
{
    const int p0 = h->parity;
    if (h->step_graph[p0]) return h->step_graph[p0];
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int k = 0; k < kStepGraph && e == cudaSuccess; ++k) {
            e = lbmp::launch_step(h);
            h->parity ^= 1;
            lbmp::sync_aa(h);
        }
        h->parity = p0;
        lbmp::sync_aa(h);
        const cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->step_graph[p0], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        cudaGetLastError();
        h->step_graph[p0] = nullptr;
        h->graph_off = true;  // plain launches from now on
        return nullptr;
    }
    return h->step_graph[p0];
}

}  // namespace

extern "C" {

const char* lbmp_last_error(void) { return g_msg; }

int lbmp_create(const lbmp_grid* grid, lbmp_lattice lattice, const lbmp_params* params, void* cuda_stream,
                lbmp_handle** out)
{
    return lbmp_create_ex(grid, lattice, params, cuda_stream, nullptr, out);
}

int lbmp_create_ex(const lbmp_grid* grid, lbmp_lattice lattice, const lbmp_params* params, void* cuda_stream,
                   const lbmp_allocator* allocator, lbmp_handle** out)
{
    if (allocator && (!allocator->alloc || !allocator->free))
        return fail(LBMP_ERR_INVALID_ARG, "allocator needs both alloc and free");
    if (!grid || !params || !out) return fail(LBMP_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (lattice != LBMP_D2Q9 && lattice != LBMP_D3Q27) return fail(LBMP_ERR_INVALID_ARG, "unknown lattice");
    const int D = (lattice == LBMP_D3Q27) ? 3 : 2;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return fail(LBMP_ERR_INVALID_ARG, "grid sizes must be >= 1");
    if (D == 2 && grid->nz != 1) return fail(LBMP_ERR_INVALID_ARG, "D2Q9 needs nz = 1");
    if (D == 3 && (grid->nx < 2 || grid->ny < 2 || grid->nz < 2))
        return fail(LBMP_ERR_INVALID_ARG, "D3Q27 needs every size >= 2");
    if (D == 2 && (grid->nx < 2 || grid->ny < 2)) return fail(LBMP_ERR_INVALID_ARG, "D2Q9 needs nx, ny >= 2");
    const bool sym_x = D == 2 && grid->periodic[0] == 2;
    for (int k = 0; k < D - 1; ++k)
        if (grid->periodic[k] != 1 && !(k == 0 && sym_x))
            return fail(LBMP_ERR_INVALID_ARG, "horizontal axes must be periodic (or, in 2-D, x a symmetry axis: 2)");
    if (grid->periodic[D - 1] != 0 && grid->periodic[D - 1] != 1)
        return fail(LBMP_ERR_INVALID_ARG, "the vertical axis is periodic (1) or walled (0)");
    const long long N = (long long)grid->nx * grid->ny * grid->nz;
    if (N > (1LL << 31) - 1) return fail(LBMP_ERR_INVALID_ARG, "more than 2^31-1 cells");
    if (params->storage != LBMP_FP32 && params->storage != LBMP_FP16_SHIFTED && params->storage != LBMP_BF16_SHIFTED)
        return fail(LBMP_ERR_INVALID_ARG, "unknown storage form");
    // the D3Q27 16-bit kernel stages codes as 32-bit words holding two
    // neighbouring cells; the D2Q9 one loads 2-byte codes but keeps the same rule
    if (params->storage != LBMP_FP32 && (grid->nx & 1))
        return fail(LBMP_ERR_INVALID_ARG, "16-bit storage needs an even nx");
    if (params->flags & ~63u) return fail(LBMP_ERR_INVALID_ARG, "unknown flag bits");
    if ((params->flags & LBMP_FLAG_AA) &&
        (D != 3 || params->storage != LBMP_FP32 || (params->flags & (LBMP_FLAG_PHASE_REDUCED | LBMP_FLAG_DIVU))))
        return fail(LBMP_ERR_UNSUPPORTED, "in-place AA storage needs D3Q27, FP32, the full phase lattice, no LBMP_FLAG_DIVU");
    if ((params->flags & LBMP_FLAG_DIVU) &&
        (params->storage != LBMP_FP32 || (params->flags & LBMP_FLAG_PHASE_REDUCED)))
        return fail(LBMP_ERR_UNSUPPORTED, "the divergence term needs FP32 storage and the full phase lattice");
    if ((params->flags & LBMP_FLAG_PHASE_REDUCED) && params->storage != LBMP_FP32)
        return fail(LBMP_ERR_UNSUPPORTED, "the reduced phase lattice is stored in FP32 only");
    if (sym_x && (params->storage != LBMP_FP32 || (params->flags & LBMP_FLAG_DIVU)))
        return fail(LBMP_ERR_UNSUPPORTED, "a symmetry axis needs FP32 storage and no LBMP_FLAG_DIVU");
    // the fused FP32 kernels address each population array by 32-bit byte offsets
    if (params->storage == LBMP_FP32 && !(params->flags & LBMP_FLAG_AA) && N > (1LL << 30) - 1)
        return fail(LBMP_ERR_UNSUPPORTED, "an FP32 domain with two population sets holds at most 2^30-1 cells");

    lbmp_handle* h = new (std::nothrow) lbmp_handle();
    if (!h) return fail(LBMP_ERR_NOMEM, "host allocation failed");
    memset(h, 0, sizeof *h);
    h->grid = *grid;
    h->D = D;
    h->Q = (D == 3) ? 27 : 9;
    h->reduced = (params->flags & LBMP_FLAG_PHASE_REDUCED) != 0;
    h->divu = (params->flags & LBMP_FLAG_DIVU) != 0;
    h->aa = (params->flags & LBMP_FLAG_AA) != 0;
    h->Qg = h->reduced ? 2 * D + 1 : h->Q;
    h->params = *params;
    h->N = N;
    h->stream = (cudaStream_t)cuda_stream;
    if (allocator) h->alloc = *allocator;
    int rc = derive(*params, D, h->der);
    if (rc != LBMP_OK) {
        delete h;
        return rc;
    }
    const double tau_min = 3.0 * fmin(h->der.nu_h, h->der.nu_l) + 0.5;
    if (!(tau_min > 0.5)) {
        delete h;
        return fail(LBMP_ERR_INVALID_ARG, "viscosities must be > 0");
    }
    fill_devparams(h);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "cudaGetDevice");
    }
    const size_t pop = lbmp::set_bytes(h), gpop = lbmp::gset_bytes(h);
    for (int k = 0; k < (h->aa ? 1 : 2); ++k) {
        e = lbmp::dev_alloc(h, (void**)&h->f[k], pop);
        if (e == cudaSuccess) e = lbmp::dev_alloc(h, (void**)&h->g[k], gpop);
        if (e != cudaSuccess) break;
    }
    if (h->aa) {  // one set, updated in place; phi from a pass of its own
        h->f[1] = h->f[0];
        h->g[1] = h->g[0];
        if (e == cudaSuccess) e = lbmp::ensure_phi(h);
        lbmp::sync_aa(h);
    }
    if (e == cudaSuccess && h->reduced) e = lbmp::dev_alloc(h, (void**)&h->phiu, lbmp::phiu_bytes(h));
    for (int k = 0; k < 2 && e == cudaSuccess && h->divu; ++k)
        e = lbmp::dev_alloc(h, (void**)&h->uvel[k], lbmp::uvel_bytes(h));
    // the divergence-term variant always runs the reference pair, which reads phi
    if (e == cudaSuccess && h->divu) e = lbmp::ensure_phi(h);
    h->red_blocks = 1024;
    if (e == cudaSuccess) e = lbmp::dev_alloc(h, (void**)&h->red, sizeof(double) * 4 * h->red_blocks);
    if (e == cudaSuccess) e = lbmp::dev_alloc(h, (void**)&h->red_out, red_out_bytes(h));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->red_out, 0, sizeof(double) * 16, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) h->dp.status = (int*)(h->red_out + kStatusSlot);
    if (e != cudaSuccess) {
        free_handle(h);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? fail(LBMP_ERR_NOMEM, "device allocation failed")
                                              : cuda_fail(e, "cudaMalloc");
    }
    for (int k = 0; k < 3; ++k) h->probe[k] = (k < D) ? ((&grid->nx)[k] / 2) : 0;
    h->kernel = 0;
    *out = h;
    return LBMP_OK;
}

int lbmp_destroy(lbmp_handle* h)
{
    if (!h) return LBMP_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_handle(h);
    return LBMP_OK;
}

int lbmp_get_derived(const lbmp_handle* h, lbmp_derived* out)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!out) return fail(LBMP_ERR_INVALID_ARG, "null output");
    *out = h->der;
    return LBMP_OK;
}

int lbmp_set_option(lbmp_handle* h, int option, long value)
{
    int rc = check_handle(h);
    if (rc) return rc;
    switch (option) {
    case LBMP_OPT_KERNEL:
        if (value < 0 || value > 2) return fail(LBMP_ERR_INVALID_ARG, "kernel must be 0, 1 or 2");
        if ((h->slab || h->aa) && value != 0)
            return fail(LBMP_ERR_UNSUPPORTED, "z-slabs and in-place AA storage run the fused kernel only");
        if (value == 1) {  // the reference pair keeps phi in an array of its own
            const cudaError_t e = lbmp::ensure_phi(h);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return e == cudaErrorMemoryAllocation ? fail(LBMP_ERR_NOMEM, "device allocation failed")
                                                      : cuda_fail(e, "phi array");
            }
        }
        h->kernel = (int)value;
        return LBMP_OK;
    case LBMP_OPT_CHUNK:
        if (value < 0 || value > (1L << 30)) return fail(LBMP_ERR_INVALID_ARG, "chunk must be >= 0");
        h->opt_chunk = (int)value;
        return LBMP_OK;
    case LBMP_OPT_CTAS_PER_SM:
        if (value < 0 || value > 64) return fail(LBMP_ERR_INVALID_ARG, "CTAs per SM must lie in [0, 64]");
        h->opt_ctas = (int)value;
        return LBMP_OK;
    case LBMP_OPT_TILE:
        if (value < 0 || value > 2) return fail(LBMP_ERR_INVALID_ARG, "tile must be 0, 1 or 2");
        h->opt_tile = (int)value;
        return LBMP_OK;
    case LBMP_OPT_WAIT_LIMIT_NS:
        if (value < 1000 || value > 60000000000L) return fail(LBMP_ERR_INVALID_ARG, "wait limit must lie in [1 us, 60 s]");
        h->dp.wait_ns = (unsigned long long)value;
        return LBMP_OK;
    case LBMP_OPT_TEST_POISON: {
        if (value != 1) return fail(LBMP_ERR_INVALID_ARG, "test poison must be 1");
        if (h->aa) return fail(LBMP_ERR_UNSUPPORTED, "in-place AA storage has no second population set to poison");
        const int d = 1 - h->parity;
        LBMP_CUDA(cudaMemsetAsync(h->f[d], 0xFF, lbmp::set_bytes(h), h->stream), "poison");
        LBMP_CUDA(cudaMemsetAsync(h->g[d], 0xFF, lbmp::gset_bytes(h), h->stream), "poison");
        return LBMP_OK;
    }
    case LBMP_OPT_TEST_STALL:
        if (value < 0 || value > 1) return fail(LBMP_ERR_INVALID_ARG, "test stall must be 0 or 1");
        h->dp.test_extra_tx = value ? 16u : 0u;
        return LBMP_OK;
    default:
        return fail(LBMP_ERR_INVALID_ARG, "unknown option");
    }
}

int lbmp_init(lbmp_handle* h, int case_id, const double* case_args, int nargs, unsigned long long seed)
{
    int rc = check_handle(h);
    if (rc) return rc;
    static const int need[7] = {3, 3, 3, 1, 4, 2, 5};
    if (case_id < 0 || case_id > 6) return fail(LBMP_ERR_INVALID_ARG, "unknown case");
    if (nargs < need[case_id] || (nargs > 0 && !case_args)) return fail(LBMP_ERR_INVALID_ARG, "too few case arguments");
    double a[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < nargs && k < 8; ++k) {
        if (!isfinite(case_args[k])) return fail(LBMP_ERR_INVALID_ARG, "non-finite case argument");
        a[k] = case_args[k];
    }
    if (case_id == LBMP_CASE_DROP_STATIC && !(a[0] > 0.0)) return fail(LBMP_ERR_INVALID_ARG, "radius must be > 0");
    h->parity = 0;
    lbmp::sync_aa(h);
    h->step = 0;
    for (int k = 0; k < 3; ++k) h->probe[k] = (k < h->D) ? ((&h->grid.nx)[k] / 2) : 0;
    if (case_id == LBMP_CASE_DROP_SHEET) {
        const double zc = a[1] + 0.5 * a[0] + 2.0 * h->der.W;
        int pv = (int)floor(zc + 0.5);
        const int nv = (&h->grid.nx)[h->D - 1];
        h->probe[h->D - 1] = pv < 0 ? 0 : (pv >= nv ? nv - 1 : pv);
    }
    LBMP_CUDA(cudaMemsetAsync(h->red_out + kStatusSlot, 0, sizeof(double), h->stream), "status reset");
    LBMP_CUDA(lbmp::launch_init(h, case_id, a, nargs, seed), "init kernel");
    LBMP_CUDA(lbmp::launch_mass(h, h->red_out + 12), "reference mass");
    return LBMP_OK;
}

int lbmp_step(lbmp_handle* h, long n)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (n < 0) return fail(LBMP_ERR_INVALID_ARG, "negative step count");
    if (h->slab && n > 1) return fail(LBMP_ERR_INVALID_ARG, "a z-slab takes one step at a time (ghosts are exchanged in between)");
    const bool graphs = n >= kStepGraph && step_graph_usable(h);
    if (graphs) check_graph_key(h);
    long k = 0;
    while (k < n) {
        if (graphs && h->graph_warm && n - k >= kStepGraph) {
            cudaGraphExec_t g = step_graph(h);
            if (g) {
                cudaError_t e = cudaGraphLaunch(g, h->stream);
                if (e != cudaSuccess) return cuda_fail(e, "step graph");
                h->step += kStepGraph;
                k += kStepGraph;
                continue;
            }
        }
        h->dp.step = (unsigned)h->step;
        cudaError_t e = lbmp::launch_step(h);
        if (e != cudaSuccess) return cuda_fail(e, "step kernel");
        h->parity ^= 1;
        lbmp::sync_aa(h);
        h->step += 1;
        h->graph_warm = true;
        ++k;
    }
    return LBMP_OK;
}

int lbmp_sync(lbmp_handle* h)
{
    int rc = check_handle(h);
    if (rc) return rc;
    LBMP_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    int word = 0;
    LBMP_CUDA(cudaMemcpy(&word, h->red_out + kStatusSlot, sizeof word, cudaMemcpyDeviceToHost), "status word");
    return status_of(word);
}

int lbmp_observables(lbmp_handle* h, lbmp_obs* out)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!out) return fail(LBMP_ERR_INVALID_ARG, "null output");
    const int nv = (h->D == 3) ? h->grid.nz : h->grid.ny;
    // a z-slab reduces over its own planes; probes and tips need the whole domain
    LBMP_CUDA(h->slab ? lbmp::launch_mass(h, h->red_out) : lbmp::launch_observables(h, h->red_out),
              "observables kernels");
    double* host = new (std::nothrow) double[16 + 2 * (size_t)nv];
    if (!host) return fail(LBMP_ERR_NOMEM, "host allocation failed");
    cudaError_t e = cudaMemcpyAsync(host, h->red_out, sizeof(double) * (16 + 2 * (size_t)nv), cudaMemcpyDeviceToHost,
                                    h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        delete[] host;
        return cuda_fail(e, "observables copy");
    }
    memset(out, 0, sizeof *out);
    out->mass = host[0];
    out->kinetic_energy = host[1];
    out->max_u = host[2];
    out->health = (host[3] != 0.0 ? 1 : 0) | (!(out->max_u <= kMaxSpeed) ? 2 : 0);
    out->p_in = host[4];
    out->p_out = host[5];
    out->laplace_dp = out->p_in - out->p_out;
    const double m0 = host[12];  // mass recorded on the device by lbmp_init / lbmp_set_state
    out->mass_drift_rel = (m0 != 0.0) ? (out->mass - m0) / m0 : 0.0;
    // phi = 1/2 crossings: spike = lowest on the centre column, bubble = highest on the origin column
    const double* cs = host + 16;
    const double* cb = host + 16 + nv;
    out->tip_spike = -1.0;
    for (int k = 0; k < nv; ++k)
        if (cs[k] >= 0.5) {
            out->tip_spike = (k == 0) ? 0.0 : k - (cs[k] - 0.5) / (cs[k] - cs[k - 1]);
            break;
        }
    out->tip_bubble = -1.0;
    for (int k = nv - 1; k >= 0; --k)
        if (cb[k] < 0.5) {
            out->tip_bubble = (k == nv - 1) ? (double)k : k + (0.5 - cb[k]) / (cb[k + 1] - cb[k]);
            break;
        }
    if (h->slab) {
        const double nan = std::numeric_limits<double>::quiet_NaN();
        out->p_in = out->p_out = out->laplace_dp = out->tip_spike = out->tip_bubble = nan;
    }
    out->step = h->step;
    int word = 0;
    memcpy(&word, host + kStatusSlot, sizeof word);
    delete[] host;
    rc = status_of(word);
    if (rc != LBMP_OK) return rc;
    if (out->health & 1) return fail(LBMP_ERR_UNSTABLE, "non-finite values in the state");
    if (out->health & 2) return fail(LBMP_ERR_UNSTABLE, "speed above 0.35: the run is unstable");
    return LBMP_OK;
}

int lbmp_get_state(lbmp_handle* h, double* f, double* g, double* phi)
{
    int rc = check_handle(h);
    if (rc) return rc;
    const size_t n = (size_t)h->Q * (size_t)h->N, ng = (size_t)h->Qg * (size_t)h->N;
    double *df = nullptr, *dg = nullptr;
    cudaError_t e = cudaSuccess;
    if (f) e = cudaMallocAsync(&df, n * sizeof(double), h->stream);
    if (e == cudaSuccess && g) e = cudaMallocAsync(&dg, ng * sizeof(double), h->stream);
    if (e == cudaSuccess) e = lbmp::launch_get_state(h, df, dg);
    if (e == cudaSuccess && f) e = cudaMemcpyAsync(f, df, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && g) e = cudaMemcpyAsync(g, dg, ng * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (df) cudaFreeAsync(df, h->stream);
    if (dg) cudaFreeAsync(dg, h->stream);
    if (e == cudaSuccess && phi) {
        e = lbmp::launch_phi_pass(h);
        float* tmp = new (std::nothrow) float[2 * h->N];
        if (!tmp) return fail(LBMP_ERR_NOMEM, "host allocation failed");
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tmp, lbmp::phi_buf(h), 2 * sizeof(float) * h->N, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e == cudaSuccess)
            for (long long i = 0; i < h->N; ++i) phi[i] = (double)tmp[i] + (double)tmp[h->N + i];
        delete[] tmp;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "get_state");
    return LBMP_OK;
}

int lbmp_set_state(lbmp_handle* h, const double* f, const double* g)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!f || !g) return fail(LBMP_ERR_INVALID_ARG, "null state array");
    const size_t n = (size_t)h->Q * (size_t)h->N, ng = (size_t)h->Qg * (size_t)h->N;
    double *df = nullptr, *dg = nullptr;
    cudaError_t e = cudaMallocAsync(&df, n * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&dg, ng * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(df, f, n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dg, g, ng * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->red_out + kStatusSlot, 0, sizeof(double), h->stream);
    if (e == cudaSuccess) e = lbmp::launch_set_state(h, df, dg);
    if (e == cudaSuccess) e = lbmp::launch_mass(h, h->red_out + 12);
    if (df) cudaFreeAsync(df, h->stream);
    if (dg) cudaFreeAsync(dg, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "set_state");
    return LBMP_OK;
}

size_t lbmp_state_bytes(const lbmp_handle* h)
{
    if (!h) return 0;
    return lbmp::set_bytes(h) + lbmp::gset_bytes(h) + lbmp::phiu_bytes(h) + lbmp::uvel_bytes(h);
}

int lbmp_upload(lbmp_handle* h, const void* host, size_t bytes)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!host || bytes != lbmp_state_bytes(h)) return fail(LBMP_ERR_INVALID_ARG, "bad upload size");
    const size_t nf = lbmp::set_bytes(h), ng = lbmp::gset_bytes(h), nu = lbmp::phiu_bytes(h);
    const char* src = (const char*)host;
    LBMP_CUDA(cudaMemcpyAsync(h->f[h->parity], src, nf, cudaMemcpyHostToDevice, h->stream), "upload f");
    LBMP_CUDA(cudaMemcpyAsync(h->g[h->parity], src + nf, ng, cudaMemcpyHostToDevice, h->stream), "upload g");
    if (nu) LBMP_CUDA(cudaMemcpyAsync(h->phiu, src + nf + ng, nu, cudaMemcpyHostToDevice, h->stream), "upload phi u");
    const size_t nv = lbmp::uvel_bytes(h);
    if (nv)
        LBMP_CUDA(cudaMemcpyAsync(h->uvel[h->parity], src + nf + ng + nu, nv, cudaMemcpyHostToDevice, h->stream),
                  "upload u");
    return LBMP_OK;
}

int lbmp_download(lbmp_handle* h, void* host, size_t bytes)
{
    int rc = check_handle(h);
    if (rc) return rc;
    if (!host || bytes != lbmp_state_bytes(h)) return fail(LBMP_ERR_INVALID_ARG, "bad download size");
    const size_t nf = lbmp::set_bytes(h), ng = lbmp::gset_bytes(h), nu = lbmp::phiu_bytes(h);
    char* dst = (char*)host;
    LBMP_CUDA(cudaMemcpyAsync(dst, h->f[h->parity], nf, cudaMemcpyDeviceToHost, h->stream), "download f");
    LBMP_CUDA(cudaMemcpyAsync(dst + nf, h->g[h->parity], ng, cudaMemcpyDeviceToHost, h->stream), "download g");
    if (nu) LBMP_CUDA(cudaMemcpyAsync(dst + nf + ng, h->phiu, nu, cudaMemcpyDeviceToHost, h->stream), "download phi u");
    const size_t nv = lbmp::uvel_bytes(h);
    if (nv)
        LBMP_CUDA(cudaMemcpyAsync(dst + nf + ng + nu, h->uvel[h->parity], nv, cudaMemcpyDeviceToHost, h->stream),
                  "download u");
    return LBMP_OK;
}

}  // extern "C"
