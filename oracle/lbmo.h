/*
 * lbmo.h -- plain FP64 CPU oracle of the multiphase lattice Boltzmann step of
 * Hosseini, Safari & Thevenin, "Lattice Boltzmann solver for multi-phase
 * flows: application to high Weber and Reynolds numbers" (arXiv 2101.06769).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA library
 * against the paper.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library; the two agree only on the exchange
 * format documented below (canonical direction order and array layout).
 *
 * Exchange format (an interface both sides implement independently):
 *   direction index  a = (cx+1) + 3*(cy+1) + 9*(cz+1)   (D2Q9: cz = 0, Q = 9)
 *   opposite(a)      = Q-1-a
 *   arrays           [a][z][y][x], x fastest; cell index x + nx*(y + ny*z)
 *   state            post-streaming populations f'(x,t) and g(x,t) of Sec. 2.2/2.3
 *   reduced phase lattice (LBMO_FLAG_PHASE_REDUCED): g lives on the rest and
 *                    face directions only (D3Q7 / D2Q5), in the same relative
 *                    order, r = 0..Qg-1, opposite(r) = Qg-1-r
 *
 * Parity status: every function below is pinned by tests under tests/
 * (lattice moments, finite-difference exactness, cumulant relations against
 * the general moment-cumulant formula, mass conservation, rest state,
 * moment identities, shear-wave decay, flat-interface profile, Laplace law,
 * layered Poiseuille flow, splitmix64 published outputs; for the reduced
 * phase lattice: isotropy, equilibrium and update moments, Galilean
 * invariance of an advected interface, mass, Laplace law).
 */
#ifndef LBMO_H
#define LBMO_H

#ifdef __cplusplus
extern "C" {
#endif

/* initial-condition cases.  The paper does not give its initial states; both
 * implementations take phi = (1 + tanh(2 d / W)) / 2 with d the signed
 * distance into the heavy fluid (RT: d = z - h(x, y), heavy on top;
 * drop and sheet: the larger of the drop's and the sheet's d), u = 0 except
 * the falling drop (u = -U0 in its phi-weighted region), p_h = 0 or the
 * optional hydrostatic / Laplace start, f' = f'_eq(p_h, rho, u) and
 * g = g_eq(phi, u), plus optional seeded velocity noise. */
enum {
    LBMO_CASE_RT = 0,          /* args: h0, amplitude, noise [, hydrostatic] */
    LBMO_CASE_DROP_STATIC = 1, /* args: R, p_init(0/1), noise                */
    LBMO_CASE_FLAT = 2,        /* args: x0, x1, noise   (heavy slab x0<x<x1)  */
    LBMO_CASE_POISEUILLE = 3,  /* args: noise           (heavy lower half)   */
    LBMO_CASE_DROP_SHEET = 4,  /* args: D, sheet_h, U0, noise [, axis]: the drop's
                                  horizontal axis coordinate (default n/2) */
    LBMO_CASE_SHEAR_WAVE = 5,  /* args: U, noise        (phi = 1)            */
    LBMO_CASE_UNIFORM = 6      /* args: phi0, p0, ux, uy, uz                 */
};

/* switches for readings where the paper admits an alternative */
enum {
    LBMO_FLAG_WE_LIGHT = 1u << 0,      /* We built on rho_l instead of rho_h        */
    LBMO_FLAG_DYNAMIC_VISC = 1u << 1,  /* interpolate eta linearly, nu = eta/rho     */
    LBMO_FLAG_UNIFORM_FORCE = 1u << 2, /* body force = force_x along x (no gravity)  */
    /* phase field on D3Q7 / D2Q5 with the first-order equilibrium and the
     * correction term C_bar of Sec. 2.2 (instead of the second-order
     * equilibrium on the flow lattice) */
    LBMO_FLAG_PHASE_REDUCED = 1u << 3,
    /* keep the w cs2 rho div(u) term of Xi (Sec. 2.3) with div(u) the
     * isotropic difference of the previous step's velocity (alternative to
     * reading A6, which drops it) */
    LBMO_FLAG_DIVU = 1u << 4
};

typedef struct {
    double rho_ratio, nu_ratio; /* rho_h/rho_l, nu_l/nu_h (rho_h = 1)                 */
    double We, Re, atwood;      /* atwood > 0 overrides rho_ratio                     */
    double mobility, width;     /* M, W                                               */
    double g_accel, U0, L_ref;  /* gravity along -vertical, impact speed, length      */
    double sigma, nu_h;         /* >= 0 / > 0: explicit values, else derived          */
    double force_x;             /* uniform force density (LBMO_FLAG_UNIFORM_FORCE)    */
    unsigned flags;
} lbmo_phys;

typedef struct {
    double rho_h, rho_l, nu_h, nu_l, sigma, beta, kappa;
    double M, W, tau_phi, lambda_phi, g_accel, U_ref, force_x;
    double K_impact;            /* We^(1/2) Re^(1/4), Sec. 3.4                        */
} lbmo_derived;

typedef struct {
    double mass, kinetic_energy, max_u, p_in, p_out, laplace_dp;
    double tip_spike, tip_bubble;
    long step;
    int health;
} lbmo_obs;

typedef struct lbmo lbmo;

/* dims = {nx, ny, nz} (nz = 1 for D = 2); periodic = {px, py, pz}, 1 = periodic,
 * 0 = half-way bounce-back walls at both ends of that axis, 2 = a symmetry
 * axis (horizontal axes only, not with LBMO_FLAG_DIVU): half-way specular
 * reflection at both of its faces, the phi ghost equal to the boundary cell
 * (reading A28).  Returns NULL on invalid input (message via lbmo_last_error). */
lbmo *lbmo_create(int D, const int dims[3], const int periodic[3], const lbmo_phys *p);
void lbmo_destroy(lbmo *s);
const char *lbmo_last_error(void);
int lbmo_derive(int D, const lbmo_phys *p, lbmo_derived *out);
void lbmo_get_derived(const lbmo *s, lbmo_derived *out);

/* relaxation rates of the general cumulant path: shear (<=0: from viscosity),
 * bulk, 3rd..6th order.  Defaults: shear from nu, all others 1 (Sec. 2.3). */
void lbmo_set_rates(lbmo *s, double shear, double bulk, double r3, double r4, double r5, double r6);

int lbmo_init(lbmo *s, int case_id, const double *args, int nargs, unsigned long long seed);
void lbmo_step(lbmo *s, long n);
void lbmo_get_state(const lbmo *s, double *f, double *g, double *phi);
void lbmo_set_state(lbmo *s, const double *f, const double *g);
void lbmo_observables(const lbmo *s, lbmo_obs *out);
/* per-cell macroscopic fields: rho, p_h, u[D] -> arrays of size N each (u: D*N) */
void lbmo_fields(const lbmo *s, double *rho, double *p, double *u);
void lbmo_set_threads(int n);
int lbmo_get_threads(void);

/* ---- pieces exposed for the pin tests ---- */
void lbmo_lattice(int D, int *Q, int *c /* Q*3 */, double *w /* Q */);
/* lattice of the phase field: the flow lattice (reduced = 0) or D3Q7 / D2Q5
 * (reduced = 1); cs2 = its squared sound speed */
void lbmo_phase_lattice(int D, int reduced, int *Q, int *c /* Q*3 */, double *w /* Q */, double *cs2);
/* isotropic finite differences (Sec. 2.2) of an arbitrary field on the grid of s */
void lbmo_fd(const lbmo *s, const double *field, double *grad /* 3*N */, double *lap /* N */);
/* central moments (27, index a + 3b + 9c) of populations h about velocity u */
void lbmo_central_moments(int D, const double *h, const double u[3], double *kappa);
void lbmo_cumulants_forward(int D, const double *kappa, double *K);
void lbmo_cumulants_inverse(int D, const double *K, double *kappa);
void lbmo_kron_inverse(int D, const double *kappa, const double u[3], double *h);
/* one cell of the collision (Sec. 2.2 and 2.3), everything in FP64.
 * diag (may be NULL) receives: rho, u[3], p_h, theta, omega, F[3], sumXi, sumcXi[3] */
void lbmo_collide_cell(const lbmo *s, const double *f, const double *g, double phi,
                       const double grad[3], double lap, double *fout, double *gout, double *diag);
/* the same with the previous step's phi u of the cell (reduced phase lattice:
 * d/dt(phi u) = phi u - phiu_prev; NULL = 0).  diag (size >= 17) also
 * receives this step's phi u at diag[14..16]. */
void lbmo_collide_cell_prev(const lbmo *s, const double *f, const double *g, double phi, const double grad[3],
                            double lap, const double *phiu_prev, double *fout, double *gout, double *diag);
/* the same with div(u) for the w cs2 rho div(u) term of Xi (LBMO_FLAG_DIVU) */
void lbmo_collide_cell_ex(const lbmo *s, const double *f, const double *g, double phi, const double grad[3],
                          double lap, const double *phiu_prev, double divu, double *fout, double *gout, double *diag);
/* number of phase-field populations of s (Qg) */
int lbmo_phase_q(const lbmo *s);
/* div(u) = (1/cs2) sum_a w_a c_a . u(x + c_a) of a velocity field u ([k][cell],
 * k < 3) on the grid of s; across a wall the ghost velocity is minus the wall
 * cell's (no slip), elsewhere periodic */
void lbmo_divu(const lbmo *s, const double *u, double *div);
unsigned long long lbmo_splitmix64(unsigned long long seed, unsigned long long counter);

#ifdef __cplusplus
}
#endif
#endif
