/*
 * lbmp.h -- C ABI of the GB300 (sm_103a) multiphase lattice Boltzmann step.
 *
 * The library advances the coupled update of Hosseini, Safari & Thevenin,
 * "Lattice Boltzmann solver for multi-phase flows: application to high Weber
 * and Reynolds numbers" (arXiv 2101.06769):
 *   - the conservative Allen-Cahn phase-field populations g (Sec. 2.2:
 *     second-order equilibrium, sharpening source, BGK relaxation with
 *     tau_phi = M/cs2, phi = sum g, isotropic finite differences);
 *   - the pressure-based hydrodynamic populations f' (Sec. 2.3: modified
 *     distribution, source Xi with pressure, surface-tension and body forces,
 *     pre-conditioning, collision in cumulant space with the shear rate on
 *     the second-order cumulants and unit rates elsewhere), with the density
 *     interpolated linearly from phi (Sec. 2.3) and the viscosity
 *     interpolated from phi (not stated in the paper: linear kinematic by
 *     default, linear dynamic with LBMP_FLAG_DYNAMIC_VISC).
 * Every step of the update runs in hand-written CUDA kernels; there is no CPU
 * fallback.  All entry points return LBMP_OK (0) or a negative status and
 * never throw; lbmp_last_error() describes the last failure of the calling
 * thread.
 *
 * Exchange format shared with external code (get/set state):
 *   direction a = (cx+1) + 3*(cy+1) + 9*(cz+1) with c in {-1,0,1}^D
 *   (D2Q9: cz = 0, Q = 9; D3Q27: Q = 27), opposite(a) = Q-1-a;
 *   arrays [a][z][y][x] with x fastest; FP64; the state is the post-streaming
 *   population set f'(x,t), g(x,t) of Sec. 2.2/2.3.
 *
 * Geometry: horizontal axes (x, and y in 3-D) are periodic; the vertical
 * axis (y in 2-D, z in 3-D) is periodic or closed by half-way bounce-back
 * no-slip walls (Sec. 3.2).  Gravity acts along -vertical.
 */
#ifndef LBMP_H
#define LBMP_H

#include <stddef.h>

#if defined(__GNUC__)
#define LBMP_API __attribute__((visibility("default")))
#else
#define LBMP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { LBMP_D2Q9 = 0, LBMP_D3Q27 = 1 } lbmp_lattice;

/* population storage: FP32, or FP16/BF16 scaled deviations from a reference
 * state decoded to FP32 in registers (arithmetic is FP32 in every form) */
typedef enum { LBMP_FP32 = 0, LBMP_FP16_SHIFTED = 1, LBMP_BF16_SHIFTED = 2 } lbmp_storage;

enum {
    LBMP_OK = 0,
    LBMP_ERR_INVALID_ARG = -1,
    LBMP_ERR_NOMEM = -2,
    LBMP_ERR_CUDA = -3,
    LBMP_ERR_TIMEOUT = -4,
    LBMP_ERR_UNSTABLE = -5,
    LBMP_ERR_UNSUPPORTED = -6
};

/* initial conditions of lbmp_init (tanh profiles phi = (1 + tanh(2d/W))/2
 * with d the signed distance into the heavy fluid; u = 0 unless stated;
 * f' = f'_eq(p_h, rho, u), g = g_eq(phi, u)).  "noise" adds a seeded uniform
 * velocity perturbation of amplitude noise * U_ref * phi per component, drawn
 * from splitmix64(seed, 3*cell + component). */
enum {
    LBMP_CASE_RT = 0,          /* args: h0, amplitude, noise [, hydrostatic]. Heavy above
                                  h = h0 + amp [cos(2 pi x/nx) (+ cos(2 pi y/ny) in 3-D)];
                                  hydrostatic != 0 starts p_h in column-wise balance with
                                  the body force: p = -g (rho_h - rho_l)(W/4) ln cosh(2(z-h)/W) */
    LBMP_CASE_DROP_STATIC = 1, /* args: R, p_init, noise. Heavy drop of radius R at the
                                  cell (nx/2, ny/2, nz/2); p_init != 0 starts
                                  p_h = (D-1) sigma/R phi */
    LBMP_CASE_FLAT = 2,        /* args: x0, x1, noise. Heavy slab x0 < x < x1 */
    LBMP_CASE_POISEUILLE = 3,  /* args: noise. Heavy lower half of the vertical axis */
    LBMP_CASE_DROP_SHEET = 4,  /* args: D, sheet_h, U0, noise [, axis]. Heavy sheet below
                                  vertical coordinate sheet_h and a drop of diameter D
                                  centred sheet_h + D/2 + 2W above the bottom, falling at
                                  U0; its horizontal axis at n/2, or at the coordinate
                                  axis (-0.5: on the left face of a symmetry axis) */
    LBMP_CASE_SHEAR_WAVE = 5,  /* args: U, noise. phi = 1, u_x = U sin(2 pi y/ny) */
    LBMP_CASE_UNIFORM = 6      /* args: phi0, p0, ux, uy, uz */
};

/* switches for readings where the paper admits an alternative */
enum {
    LBMP_FLAG_WE_LIGHT = 1u << 0,     /* sigma = rho_l L U^2/We (the paper's printed We) */
    LBMP_FLAG_DYNAMIC_VISC = 1u << 1, /* eta(phi) linear, nu = eta/rho */
    LBMP_FLAG_UNIFORM_FORCE = 1u << 2, /* body force = force_x along x instead of gravity */
    /* Phase field on the reduced lattice D3Q7 / D2Q5 (rest and face
     * directions, weights 1/4, 1/8 and cs2 = 1/4 in 3-D; 1/3, 1/6 and
     * cs2 = 1/3 in 2-D) with the first-order equilibrium w phi (1 + c.u/cs2)
     * and the correction term (1 - 1/(2 tau)) (w/cs2) c . d/dt(phi u) of
     * Sec. 2.2, d/dt(phi u) the backward difference of a stored per-cell
     * phi u (the previous value equals the current one before the first step
     * after lbmp_init / lbmp_set_state).  The flow lattice is unchanged.
     * FP32 storage only (LBMP_ERR_UNSUPPORTED otherwise). */
    LBMP_FLAG_PHASE_REDUCED = 1u << 3,
    /* Keep the w cs2 rho div(u) term of Xi (Sec. 2.3), which the default
     * reading drops (div u prescribed zero): div(u) is the isotropic
     * difference of the previous step's velocity, stored per cell (no-slip
     * ghosts across walls; before the first step after lbmp_init /
     * lbmp_set_state the previous velocity is the current one).  An ablation
     * of that reading: the term cancels the pressure's response to the
     * divergence.  FP32 storage and the full phase lattice only
     * (LBMP_ERR_UNSUPPORTED otherwise); runs the reference pair; not a batch
     * member. */
    LBMP_FLAG_DIVU = 1u << 4,
    /* In-place AA storage (esoteric pull, Sec. 2.2 / 2.3 streaming): one
     * population set each for f' and g instead of two, half the state.
     * Even steps read every population of a cell from the cell itself and
     * write the post-collision values back to it in the opposite
     * directions' slots; odd steps read from the neighbours' opposite slots
     * and write to the neighbours' own slots; each cell touches only the
     * slots it reads, so the update is race-free in place.  phi, which the
     * two-set kernels form from the g they stage (ring cells included), is
     * formed by a separate phase-aware pass first (8 bytes per cell more
     * state; 116 bytes per cell more traffic per step), because a ring read
     * would race with the owner's in-place writes.  D3Q27, FP32 storage, the
     * full phase lattice, no LBMP_FLAG_DIVU (LBMP_ERR_UNSUPPORTED
     * otherwise); the fused kernel only (LBMP_OPT_KERNEL 0); no autotuning
     * (a trial launch would advance the state in place); not a batch member
     * or a z-slab.  lbmp_download / lbmp_upload images hold the phase of the
     * step count: upload into a handle whose step count has the same
     * parity. */
    LBMP_FLAG_AA = 1u << 5
};

typedef struct {
    int nx, ny, nz;  /* nz = 1 for D2Q9; nx even with FP16/BF16 storage; at most 2^31-1 cells,
                        2^30-1 for an FP32 domain with two population sets (the default: its
                        kernels address each population array by 32-bit byte offsets) */
    int periodic[3]; /* 1 = periodic; 0 = half-way bounce-back walls (vertical axis only);
                        2 = symmetry axis (x of a D2Q9 FP32 domain only; not with
                        LBMP_FLAG_DIVU): half-way specular reflection
                        at both faces, the phi ghost equal to the boundary cell -- the
                        symmetry boundary of the 2-D splash, Sec. 3.4 */
} lbmp_grid;

/* problem statement (lattice units, heavy density rho_h = 1, Sec. 3) */
typedef struct {
    double rho_ratio, nu_ratio; /* rho_h/rho_l, nu_l/nu_h                                  */
    double We, Re, atwood;      /* atwood > 0 overrides rho_ratio = (1+At)/(1-At)           */
    double mobility, width;     /* M, W                                                     */
    double g_accel, U0, L_ref;  /* gravity, impact speed, reference length (L_x or D)       */
    double sigma, nu_h;         /* explicit overrides: sigma >= 0, nu_h > 0; else derived:
                                   nu_h = U L/Re with U = U0 or sqrt(g L);
                                   sigma = rho_h L U^2/We (0 when We = 0)                   */
    double force_x;             /* with LBMP_FLAG_UNIFORM_FORCE                             */
    int storage;                /* lbmp_storage                                             */
    unsigned flags;             /* LBMP_FLAG_*                                              */
} lbmp_params;

/* derived lattice parameters: beta = 12 sigma/W, kappa = 3 sigma W/2 (Sec. 2.1),
 * tau_phi = M/cs2 + 1/2, lambda_phi = 1 - 1/(2 tau_phi) (Sec. 2.2) */
typedef struct {
    double rho_h, rho_l, nu_h, nu_l, sigma, beta, kappa;
    double M, W, tau_phi, lambda_phi, g_accel, U_ref, force_x;
} lbmp_derived;

/* FP64 observables (reductions on the device):
 *   mass = sum phi; mass_drift_rel = (mass - mass at lbmp_init/set_state)/that;
 *   kinetic_energy = sum rho |u|^2 / 2; max_u = max |u|;
 *   p_in/p_out = mean p_h over the 3^D block at the probe cell (drop centre) and
 *   at the origin, laplace_dp = p_in - p_out (Sec. 3.1);
 *   tip_spike = lowest phi = 1/2 crossing on the vertical column through
 *   (nx/2, ny/2), tip_bubble = highest crossing on the column through the
 *   origin (Sec. 3.2/3.3; -1 when there is none); health: bit 0 set when a
 *   non-finite value was met, bit 1 when max_u exceeds 0.35 (far beyond the
 *   low-Mach range the scheme is valid in; such a run is unstable). */
typedef struct {
    double mass, mass_drift_rel, kinetic_energy, max_u, p_in, p_out, laplace_dp;
    double tip_spike, tip_bubble;
    long step;
    int health;
} lbmp_obs;

typedef struct lbmp_handle lbmp_handle;

/* Create a domain.  cuda_stream is a cudaStream_t (NULL = legacy default
 * stream); every later call of the handle is ordered on it.  Allocates the
 * device state with cudaMalloc: two FP32/FP16/BF16 population sets for f'
 * and g, the stored previous phi u of the reduced phase lattice, the stored
 * velocities of LBMP_FLAG_DIVU, a phi field (8 bytes per cell) only for the
 * reference pair (LBMP_OPT_KERNEL = 1, or LBMP_FLAG_DIVU), and a few KiB for
 * the observables; no device work.  The fused kernels never store phi: the
 * observables and lbmp_get_state form it in the population set the next
 * step overwrites.  Errors: INVALID_ARG (bad grid or parameters), NOMEM,
 * CUDA.  The caller owns *out and releases it with lbmp_destroy. */
LBMP_API int lbmp_create(const lbmp_grid *grid, lbmp_lattice lattice, const lbmp_params *params,
                void *cuda_stream, lbmp_handle **out);

/* Caller-supplied device memory (an allocator callback, e.g. a framework's
 * caching allocator): alloc(bytes, stream, ctx) returns a device pointer to
 * at least `bytes` bytes, aligned to 256 bytes, usable on `stream` (the
 * handle's stream), or NULL when it cannot; free(ptr, bytes, stream, ctx)
 * gives it back.  Every device array a handle keeps for its lifetime comes
 * from alloc and goes back through free, at lbmp_destroy or when
 * lbmp_create_ex fails; ctx is passed through unchanged.  Both callbacks are
 * called from the thread that makes the lbmp call, never from the GPU. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, size_t bytes, void *stream, void *ctx);
    void *ctx;
} lbmp_allocator;

/* lbmp_create with the handle's device arrays from `allocator` (NULL: as
 * lbmp_create).  A NULL return of alloc fails the call with LBMP_ERR_NOMEM
 * after freeing what was already allocated. */
LBMP_API int lbmp_create_ex(const lbmp_grid *grid, lbmp_lattice lattice, const lbmp_params *params,
                            void *cuda_stream, const lbmp_allocator *allocator, lbmp_handle **out);
LBMP_API int lbmp_destroy(lbmp_handle *h);
LBMP_API const char *lbmp_last_error(void);
LBMP_API int lbmp_get_derived(const lbmp_handle *h, lbmp_derived *out);

/* Set the initial state of one of the LBMP_CASE_* problems on the device
 * (Sec. 3 set-ups; reading A18).  Asynchronous. */
LBMP_API int lbmp_init(lbmp_handle *h, int case_id, const double *case_args, int nargs,
              unsigned long long seed);

/* Advance n time steps (Sec. 2.2/2.3), asynchronously on the handle's stream.
 * With FP32 storage, n >= 16 and a stream other than the legacy default one
 * that is not itself being captured, runs of 16 steps replay a CUDA graph
 * captured once per starting parity after the first plain step (bitwise the
 * same as plain launches; recaptured when a launch option changes).  FP16/BF16 storage launches step by step: its stochastic
 * rounding of the codes is seeded with the step index.  Errors: INVALID_ARG
 * for n < 0. */
LBMP_API int lbmp_step(lbmp_handle *h, long n);

/* Wait for the handle's stream; reports a device-side error status:
 * LBMP_ERR_TIMEOUT when a bounded wait inside a step kernel ran out (the
 * kernel then stopped early and the state is invalid; re-initialise). */
LBMP_API int lbmp_sync(lbmp_handle *h);

/* FP64 observables (synchronises); LBMP_ERR_TIMEOUT as lbmp_sync,
 * LBMP_ERR_UNSTABLE when the state holds non-finite values. */
LBMP_API int lbmp_observables(lbmp_handle *h, lbmp_obs *out);

/* Host copies of the state in the exchange format (synchronise).  f holds
 * Q*N doubles, g Qg*N (Qg = Q, or 2D+1 with LBMP_FLAG_PHASE_REDUCED: the
 * rest and face directions in the same relative order, opposite(r) =
 * Qg-1-r), phi N doubles; any of them may be NULL in get_state. */
LBMP_API int lbmp_get_state(lbmp_handle *h, double *f, double *g, double *phi);
/* set_state recomputes phi and, with LBMP_FLAG_PHASE_REDUCED or
 * LBMP_FLAG_DIVU, takes the stored previous phi u / velocity equal to the
 * current ones (as lbmp_init does). */
LBMP_API int lbmp_set_state(lbmp_handle *h, const double *f, const double *g);

/* Raw transfers of the device state in its native storage layout (an opaque
 * byte image, valid only for a handle of the same grid, lattice, storage and
 * flags; with LBMP_FLAG_PHASE_REDUCED it includes the stored phi u, with
 * LBMP_FLAG_DIVU the stored velocity).  Asynchronous on the handle's
 * stream; host memory should be pinned.  bytes must equal
 * lbmp_state_bytes(h). */
LBMP_API size_t lbmp_state_bytes(const lbmp_handle *h);
LBMP_API int lbmp_upload(lbmp_handle *h, const void *host, size_t bytes);
LBMP_API int lbmp_download(lbmp_handle *h, void *host, size_t bytes);

/* Options of a handle.
 *   LBMP_OPT_KERNEL: 0 = default fused kernel (g staged by 4-byte cp.async),
 *     1 = simple reference pair (phi pass + one thread per cell), 2 = for
 *     FP32 D3Q27 with nx % 4 == 0 the fused kernel with g staged by bulk
 *     copies (TMA engine) and bounded mbarrier waits, else as 0; for A/B
 *     tests and measurement.  0 and 1 give bitwise identical results; 2
 *     performs the same operations but the compiler may fuse a multiply-add
 *     differently, so it agrees to within a few ulps.
 *   LBMP_OPT_CHUNK: planes (rows in 2-D) per work item of the fused
 *     kernels, 0 = automatic (the default), else >= 1.
 *   LBMP_OPT_CTAS_PER_SM: resident CTAs per SM of the fused kernels'
 *     persistent grid, 0 = the occupancy maximum (the default), else >= 1
 *     (values above the maximum act as the maximum).
 *   LBMP_OPT_WAIT_LIMIT_NS: bound of every wait inside a step kernel, in ns
 *     (default 2e9; range [1e3, 6e10]).
 *   LBMP_OPT_TEST_STALL (test only): 1 arms each staging barrier of the
 *     bulk-copy kernel for 16 bytes more than its copies deliver, so that its
 *     waits run out and the next lbmp_sync reports LBMP_ERR_TIMEOUT; 0 off.
 *   LBMP_OPT_TILE: tile shape of the FP32 D3Q27 fused kernel: 0 = 32 x 4
 *     (default), 1 = 16 x 8, 2 = 8 x 16.
 *   LBMP_OPT_TEST_POISON (test only): 1 fills the population set the next
 *     step writes with NaN (the step must overwrite every slot; a missed
 *     slot shows in the state).
 * CHUNK and CTAS_PER_SM change speed only, never results; each TILE value
 * is a separately compiled build of the same kernel and agrees with the
 * default to within rounding.  Returns LBMP_ERR_INVALID_ARG for an unknown
 * option or an out-of-range value. */
enum {
    LBMP_OPT_KERNEL = 0,
    LBMP_OPT_CHUNK = 1,
    LBMP_OPT_CTAS_PER_SM = 2,
    LBMP_OPT_WAIT_LIMIT_NS = 3,
    LBMP_OPT_TEST_STALL = 4,
    LBMP_OPT_TILE = 5,
    LBMP_OPT_TEST_POISON = 6
};
LBMP_API int lbmp_set_option(lbmp_handle *h, int option, long value);

/* Launch-shape autotuner of the fused step kernel (no counterpart in the
 * paper; serving-side tuning).  Times each candidate (tile shape in {32 x 4,
 * 16 x 8, 8 x 16} for the FP32 D3Q27 kernel, planes per work item -- cells
 * per thread per work item -- in {automatic, 1, 2, 4, 8, 16, 32, 64, 128} up to
 * the marching extent, CTAs per SM in {maximum, 1, 2}) over `reps` launches
 * (>= 1) after one warm-up launch, with CUDA events on the handle's stream,
 * and keeps the fastest as the handle's options.  Trial launches read the
 * current population set and write the other one, which the next step
 * overwrites: the state is not advanced.  `table` (caller-owned, may be NULL)
 * receives up to max_entries trials; *n_entries (may be NULL) the number of
 * trials run.  With LBMP_OPT_KERNEL = 1 nothing is tuned (n_entries = 0).
 * Synchronises the handle's stream. */
typedef struct {
    int chunk;        /* LBMP_OPT_CHUNK value of the trial (0 = automatic) */
    int ctas_per_sm;  /* LBMP_OPT_CTAS_PER_SM value of the trial (0 = maximum) */
    double ms;        /* mean time of one step launch */
    int tile;         /* LBMP_OPT_TILE value of the trial */
} lbmp_tune_entry;
LBMP_API int lbmp_autotune(lbmp_handle *h, int reps, lbmp_tune_entry *table, int max_entries, int *n_entries);

/* Name of the current CUDA device (for keying tuning caches); writes a
 * NUL-terminated string of at most len bytes. */
LBMP_API int lbmp_device_name(char *out, int len);

/* ---- batches: many domains advanced together ------------------------------
 * A batch advances every member domain with one persistent kernel launch per
 * lattice type and step: the kernel walks a device-side table of the members
 * (sizes, parameters, population sets, parity, steps left) and splits their
 * combined work evenly over the GPU, so small and uneven domains share the
 * machine instead of each under-filling it.  The per-step bookkeeping
 * (parity, remaining steps) is done on the device, so a run of steps is
 * captured once in a CUDA graph and replayed until the membership changes.
 * D3Q27 and D2Q9 members may be mixed (one kernel per lattice type).
 * Results are bitwise those of stepping each member alone.
 * Members are handles from lbmp_create on the batch's device; the batch does
 * not own them.  A member must not be stepped, set or destroyed through its
 * own handle while it belongs to a batch (remove it first); get_state and
 * observables of a member are valid after lbmp_batch_step returns. */
typedef struct lbmp_batch lbmp_batch;

/* hbm_budget: upper bound (bytes) on the summed device state of the members,
 * 0 = none; cuda_stream: stream of all batch work (NULL: the batch creates a
 * private stream, since the legacy default stream cannot be captured). */
LBMP_API int lbmp_batch_create(size_t hbm_budget, void *cuda_stream, lbmp_batch **out);
LBMP_API int lbmp_batch_destroy(lbmp_batch *b);
/* Admit h for `steps` more steps (> 0).  Members may be D2Q9 or D3Q27
 * domains in any storage form and with either phase lattice (each lattice,
 * storage and phase-lattice kind runs its own persistent kernel); domains
 * with LBMP_FLAG_DIVU give LBMP_ERR_UNSUPPORTED.  LBMP_ERR_NOMEM
 * when it would exceed the budget, LBMP_ERR_INVALID_ARG when h is already a
 * member or the batch is full (1024 members). */
LBMP_API int lbmp_batch_add(lbmp_batch *b, lbmp_handle *h, long steps);
LBMP_API int lbmp_batch_remove(lbmp_batch *b, lbmp_handle *h);
/* Advance every member with steps left by up to n steps (graph launches on
 * the batch's stream), then synchronise.  *n_finished (may be NULL) receives
 * the number of members whose steps ran out during this call. */
LBMP_API int lbmp_batch_step(lbmp_batch *b, long n, int *n_finished);
/* Members and their remaining steps: fills up to max entries, returns the
 * member count (or a negative status). */
LBMP_API int lbmp_batch_members(const lbmp_batch *b, lbmp_handle **members, long *steps_left, int max);

/* Autotuner of the batch kernels (no counterpart in the paper): times one
 * step of the current members' kernels (the D3Q27 and D2Q9 batch kernels,
 * no epilogue) for each D3Q27 tile shape {32 x 4, 16 x 8, 8 x 16} and
 * planes (rows) per work item {8, 16, 32, 64}, over `reps` launches after a
 * warm-up, in two passes (each shape's time the smaller of its two), and
 * keeps the fastest for the batch; the graphs are re-captured at
 * the next lbmp_batch_step.  Trial launches read each member's current
 * population set and write the other one: no member advances and results
 * are unchanged.  table / n_entries as in lbmp_autotune (entry.tile and
 * entry.chunk set, ctas_per_sm = 0).  Synchronises the batch's stream. */
LBMP_API int lbmp_batch_autotune(lbmp_batch *b, int reps, lbmp_tune_entry *table, int max_entries,
                                 int *n_entries);

/* Mass without allocation (the paper has no counterpart: this is a service
 * of the library).  For callers that cannot allocate device memory, e.g. a
 * host framework that owns every byte of device memory and hands out only
 * views into its pool, or a fixed-budget real-time loop: returns in *mass_out
 * the FP64 sum of n_values FP32 device values g_dev, the total mass
 * sum_x phi(x) when g_dev holds a phase-field population set (the total over
 * all populations of all cells does not depend on their layout).  Uses a
 * fixed 32 KiB device array compiled into the library instead of scratch
 * memory and calls no allocating routine.  At most 2^33 values (else
 * LBMP_ERR_INVALID_ARG).  Ordered on cuda_stream (NULL = legacy default
 * stream) and synchronises it.  The first call on a device looks up the
 * array's address with that device current: make it before any stream
 * capture.  Later calls outside a capture look it up again (a device reset
 * moves the array); a call on a capturing stream uses the address of the last
 * call on that device that was not, and a first call on a capturing stream
 * returns LBMP_ERR_UNSUPPORTED.  Every call on a device shares the array, so
 * calls that overlap on the GPU race: serialise them. */
LBMP_API int lbmp_mass_noalloc(const float *g_dev, long long n_values, double *mass_out, void *cuda_stream);

/* ------------------------------------------------------------ z-slabs
 * Decomposition of a D3Q27 domain into slabs along z, one per rank (the
 * paper has no counterpart: this is how the library runs one domain on
 * several GPUs).  A slab holds the global planes [z_begin, z_end) and, on
 * every face that borders another slab, two ghost planes; on a face that is
 * the domain's own wall it keeps the wall (half-way bounce-back, mirrored
 * phi).  A step updates the slab's own planes only; between steps the
 * caller moves the populations that cross each face from the neighbour's
 * boundary planes into this slab's ghost planes (lbmp_pack_planes on the
 * sender, any transport, lbmp_unpack_planes on the receiver).  With the
 * ghosts filled every step, the slabs reproduce the undivided domain
 * bitwise.
 *
 * lbmp_create_slab: grid is the whole domain (x and y periodic; z periodic
 * or walled); 0 <= z_begin < z_end <= grid->nz with at least two planes; a
 * slab must border at least one other slab.  FP32 storage and the full
 * phase lattice only, without LBMP_FLAG_DIVU (else LBMP_ERR_UNSUPPORTED).
 * lbmp_init sets the initial state at the global positions (the same
 * seeded noise as the undivided domain); lbmp_get_state / lbmp_set_state
 * exchange the local planes, ghosts included ([a][local z][y][x]);
 * lbmp_observables reduces over the slab's own planes (mass, kinetic
 * energy, max |u|; the Laplace probes and tips are NaN: sum and gather
 * them across ranks).  lbmp_step takes n = 1 only, the fused kernel only
 * (LBMP_OPT_KERNEL 0); slabs are not batch members. */
LBMP_API int lbmp_create_slab(const lbmp_grid *grid, int z_begin, int z_end, lbmp_lattice lattice,
                              const lbmp_params *params, void *cuda_stream, const lbmp_allocator *allocator,
                              lbmp_handle **out);
/* layout[0..4] = z_begin, z_end, ghost planes below, ghost planes above,
 * local nz (the planes of the local arrays); a plain domain reports
 * 0, nz, 0, 0, nz. */
LBMP_API int lbmp_slab_layout(const lbmp_handle *h, int *layout);
/* Copy n whole planes of the current population sets into the device
 * buffer dev_buf (pack) or back (unpack): plan holds n triples (set: 0 = f',
 * 1 = g; direction a in the canonical order; local plane z), and triple k
 * occupies dev_buf[k nx ny, (k+1) nx ny).  n <= 64.  Asynchronous on the
 * handle's stream; dev_buf is the caller's device memory. */
LBMP_API int lbmp_pack_planes(lbmp_handle *h, const int *plan, int n, float *dev_buf);
LBMP_API int lbmp_unpack_planes(lbmp_handle *h, const int *plan, int n, const float *dev_buf);

#ifdef __cplusplus
}
#endif
#endif
