// lbmp_internal.h -- host-side handle of the C ABI and the kernel launchers
// shared between the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include "../../include/lbmp.h"
#include "lbmp_common.cuh"

struct lbmp_handle {
    lbmp_grid grid;
    int D, Q;
    int Qg;            // phase-field populations: Q, or 2D+1 on the reduced phase lattice
    bool reduced;      // LBMP_FLAG_PHASE_REDUCED
    lbmp_params params;
    lbmp_derived der;
    lbmp::DevParams dp;
    cudaStream_t stream;
    int device;
    long long N;
    // ping-pong population sets; buffers hold post-collision values of the
    // previous step (pull streaming reads them upstream)
    float* f[2];
    float* g[2];
    // z-slab (lbmp_create_slab): global planes [slab_z0, slab_z1) held with
    // slab_ghost[0] / [1] ghost planes below / above; slab = false otherwise
    bool slab;
    int slab_z0, slab_z1, slab_ghost[2];
    // in-place AA storage (LBMP_FLAG_AA): f[1] == f[0], g[1] == g[0], and
    // parity is the phase (0 natural, 1 swapped; dp.aa = 1 + parity)
    bool aa;
    float* phi;        // reference pair only: phi = sum g as hi [0, N) + lo [N, 2N), refreshed by the phi pass
    lbmp_allocator alloc;  // caller's device allocator (alloc == null: cudaMalloc / cudaFree)
    float* phiu;       // reduced phase lattice: phi u of the previous step, [k < D][cell]; else null
    bool divu;         // LBMP_FLAG_DIVU
    float* uvel[2];    // LBMP_FLAG_DIVU: stored velocity [k < D][cell], uvel[parity] the previous step's; else null
    int parity;        // f[parity], g[parity] hold the current state
    long step;
    int kernel;        // LBMP_OPT_KERNEL: 0 default, 1 reference pair, 2 bulk-copy staging
    int opt_chunk;     // LBMP_OPT_CHUNK: planes (rows) per work item, 0 = automatic
    int opt_ctas;      // LBMP_OPT_CTAS_PER_SM: resident CTAs per SM of the grid, 0 = occupancy maximum
    int opt_tile;      // LBMP_OPT_TILE: tile shape of the FP32 D3Q27 fused kernel (0 32x4, 1 16x8, 2 8x16)
    int probe[3];
    // step graphs (lbmp_step): kStepGraph steps captured from each starting
    // parity, for the launch options in graph_key; warm once a plain step
    // ran with those options (the kernels' one-time set-up is not captured)
    cudaGraphExec_t step_graph[2];
    long long graph_key[6];
    bool graph_warm, graph_off;
    // observables scratch (partial sums per block) and result slot
    double* red;
    int red_blocks;
    double* red_out;
};

namespace lbmp {

// one member of a batch, as the batch kernels see it (device memory)
struct BatchDomain {
    DevParams p;
    float* f[2];
    float* g[2];
    float* phiu;  // reduced phase lattice: stored previous phi u; else null
    int parity, steps_left;
    int tiles_x, tiles_y, chunk, item_begin, items;
};

// Launch shape of a persistent fused kernel over `tiles` tiles marching
// through `nmarch` planes (rows in 2-D): planes per work item and grid size,
// from the handle's options or the defaults (enough items for three rounds of
// the full-occupancy grid, at least 8 planes per item: each item stages two
// planes more than it updates, so longer items win until the rounds get
// coarse; on the 128x128x512 RT workload 32 planes per item at 4 CTAs per
// SM measured 0.852 ms per step, 16 planes 0.893 ms).
struct LaunchShape {
    int chunk, nitems, grid;
};
inline LaunchShape launch_shape(const lbmp_handle* h, int tiles, int nmarch, int per_sm, int sms)
{
    if (per_sm < 1) per_sm = 1;
    const int ctas = (h->opt_ctas > 0 && h->opt_ctas < per_sm) ? h->opt_ctas : per_sm;
    const long long cap = (long long)ctas * sms;
    int chunk;
    if (h->opt_chunk > 0) {
        chunk = h->opt_chunk < nmarch ? h->opt_chunk : nmarch;
    } else {
        chunk = nmarch;
        while (chunk > 8 && (long long)tiles * ((nmarch + chunk - 1) / chunk) < 3LL * per_sm * sms) chunk /= 2;
    }
    LaunchShape L;
    L.chunk = chunk;
    L.nitems = tiles * ((nmarch + chunk - 1) / chunk);
    L.grid = (int)(L.nitems < cap ? L.nitems : cap);
    return L;
}

// bytes of one population set (f' or g) in the handle's storage form
inline size_t set_bytes(const lbmp_handle* h)
{
    const size_t N = (size_t)h->N, Q = (size_t)h->Q;
    if (h->params.storage == LBMP_FP32) return sizeof(float) * Q * N;
    return sizeof(float) * N + sizeof(unsigned short) * (Q - 1) * N;  // reference + 16-bit codes
}
// bytes of one phase-field population set (equals set_bytes but on the reduced phase lattice)
inline size_t gset_bytes(const lbmp_handle* h)
{
    if (h->reduced) return sizeof(float) * (size_t)h->Qg * (size_t)h->N;
    return set_bytes(h);
}
// bytes of the stored previous phi u (reduced phase lattice)
inline size_t phiu_bytes(const lbmp_handle* h) { return h->reduced ? sizeof(float) * h->D * (size_t)h->N : 0; }
// bytes of one stored velocity field (LBMP_FLAG_DIVU)
inline size_t uvel_bytes(const lbmp_handle* h) { return h->divu ? sizeof(float) * h->D * (size_t)h->N : 0; }

// The autotuners time real step kernels.  On the reduced phase lattice a
// step replaces the stored previous phi u in place, so a trial launch would
// leave this step's phi u where the next step expects the previous one (its
// d/dt(phi u) would read zero).  phiu_save copies the stored phi u of h into
// a fresh device buffer (*copy, null when h keeps none) on `stream`;
// phiu_restore copies it back on `stream`, waits for the copy and frees the
// buffer.
cudaError_t phiu_save(lbmp_handle* h, cudaStream_t stream, float** copy);
cudaError_t phiu_restore(lbmp_handle* h, cudaStream_t stream, float* copy);

// device memory of a handle: the caller's allocator, or cudaMalloc
cudaError_t dev_alloc(lbmp_handle* h, void** p, size_t bytes);
void dev_free(lbmp_handle* h, void* p, size_t bytes);
// where the phi pass writes phi (hi, lo; 2N floats): the handle's phi array
// when it keeps one (the reference pair reads it while writing the other
// population set), else the f' population set the next step overwrites,
// whose contents are dead between steps
inline float* phi_buf(const lbmp_handle* h) { return h->phi ? h->phi : h->f[1 - h->parity]; }
// allocate the phi array the reference pair needs (not during a capture)
cudaError_t ensure_phi(lbmp_handle* h);

// kernel launchers (return cudaError_t of the launch)
cudaError_t launch_phi_pass(lbmp_handle* h);
cudaError_t launch_phiu_reset(lbmp_handle* h);  // reduced phase lattice: previous phi u := current
cudaError_t launch_step_simple(lbmp_handle* h);
cudaError_t launch_step_fused3(lbmp_handle* h);        // FP32 D3Q27, 32 x 4 tiles
cudaError_t launch_step_fused3_t16x8(lbmp_handle* h);  // FP32 D3Q27, 16 x 8 tiles
cudaError_t launch_step_fused3_t8x16(lbmp_handle* h);  // FP32 D3Q27, 8 x 16 tiles
cudaError_t launch_step_fused3_red(lbmp_handle* h);    // FP32 D3Q27 flow, D3Q7 phase field, 32 x 4 tiles
cudaError_t launch_init(lbmp_handle* h, int case_id, const double* args, int nargs, unsigned long long seed);
cudaError_t launch_set_state(lbmp_handle* h, const double* dev_f, const double* dev_g);
cudaError_t launch_get_state(lbmp_handle* h, double* dev_f, double* dev_g);
// dev_out: [0..3] mass, kinetic energy, max|u|, non-finite count; [4..5] probe
// pressures; [16..16+2nv) phi on the spike and bubble columns
cudaError_t launch_observables(lbmp_handle* h, double* dev_out);
cudaError_t launch_mass(lbmp_handle* h, double* dev_out4);  // writes 4 doubles, [0] = mass
bool fused_supported(const lbmp_handle* h);
// batch kernel of one tile shape of the FP32 D3Q27 fused step
struct Batch3Ops {
    int tile_x, tile_y;
    cudaError_t (*prepare)(int device);  // attributes and occupancy (not capturable)
    // persistent form (null where a kind has the member-grid form): the
    // members' work items walked by one grid, members read from the device table
    cudaError_t (*launch)(const BatchDomain* table, int ndom, int nitems, int device, cudaStream_t stream);
    // member-grid form (null where a kind has none): members [0, n) of the
    // host table `host` passed as kernel parameters, each with its population
    // sets for the parity host[k].parity ^ flip; blockIdx.y selects the member,
    // whose steps_left the kernel reads from the device table `dev`.  At most
    // grid_members members per launch.
    cudaError_t (*launch_grid)(const BatchDomain* host, const BatchDomain* dev, int n, int flip, int device,
                               cudaStream_t stream);
    int grid_members;
};
extern const Batch3Ops batch3_ops_32x4, batch3_ops_16x8, batch3_ops_8x16;
extern const Batch3Ops batch3_ops_f16, batch3_ops_bf16;  // shifted 16-bit members (32 x 4 tiles)
extern const Batch3Ops batch3_ops_red;                    // FP32 members with the D3Q7 phase field
extern const Batch3Ops batch2_ops_f16, batch2_ops_bf16;  // shifted 16-bit D2Q9 members (128-cell rows)
cudaError_t launch_step_fused2s(lbmp_handle* h);         // shifted 16-bit storage, D2Q9
inline const Batch3Ops& batch3_ops(int tile)
{
    return tile == 1 ? batch3_ops_16x8 : (tile == 2 ? batch3_ops_8x16 : batch3_ops_32x4);
}
cudaError_t launch_step_fused2(lbmp_handle* h);
cudaError_t launch_step_aa(lbmp_handle* h);  // in-place AA storage: phi pass, then the AA step of the phase
// keep dp.aa in step with the phase after every change of parity
inline void sync_aa(lbmp_handle* h)
{
    if (h->aa) h->dp.aa = 1 + h->parity;
}
cudaError_t launch_step_fused16(lbmp_handle* h);  // shifted 16-bit storage, D3Q27
bool bulk_supported(const lbmp_handle* h);         // FP32 D3Q27 with nx % 4 == 0
cudaError_t launch_step_fused_bulk(lbmp_handle* h);
// the step kernel(s) selected by LBMP_OPT_KERNEL for this handle (no parity flip)
cudaError_t launch_step(lbmp_handle* h);
int batch2_tile_x();
cudaError_t prepare_batch2(int device, bool reduced, bool sym);  // reduced: D2Q5 phase field; sym: x symmetry axis
cudaError_t launch_batch2(const BatchDomain* table, int ndom, int nitems, int device, cudaStream_t stream,
                          bool reduced, bool sym);
cudaError_t launch_batch_epilogue(BatchDomain* table, int ndom, cudaStream_t stream);
// record a message for lbmp_last_error() and return code
int set_error(int code, const char* msg);

}  // namespace lbmp
