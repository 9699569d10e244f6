/*
 * lbmo.c -- plain FP64 CPU oracle of the coupled phase-field / pressure-based
 * cumulant lattice Boltzmann step (Hosseini, Safari & Thevenin, arXiv 2101.06769).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
 * baseline of the benchmark.  It is deliberately slow and literal:
 *   - every population set is a separate [a][cell] FP64 array,
 *   - streaming is a two-array push,
 *   - the flow collision goes through the full 27 central moments, the full
 *     cumulant relations (Sec. 2.3) and back, with a general rate vector,
 * so that a reader can check each step against the paper by eye.  It shares
 * no code with the CUDA library.
 *
 * Readings of the paper taken here, where it is silent, garbled or ambiguous:
 *   A1  mu_phi = 2 beta phi (phi-1)(2phi-1) - kappa lap(phi)       (Sec. 2.1)
 *   A2  force on the fluid = +F_s + F_b, F_s = mu_phi grad(phi)    (Sec. 2.3)
 *   A3  +S_bar on the right-hand side of the g update                (Sec. 2.2)
 *   A4  S_bar factor (1 - 1/(2 tau_bar_phi)), tau_bar_phi = M/cs2 + 1/2
 *   A5  g_eq normalised by density: w phi [1 + c.u/cs2 + H:uu/(2cs4)]
 *   A6  the w cs2 rho div(u) term of Xi is dropped (prescribed div u = 0)
 *   A7  omega = 1/(nu/cs2 + 1/2)
 *   A8  collide h = f^p - w(theta - 1), theta = sum f^p
 *   A9  corrected 6th-order cumulant relation (Pi_yz Pi_x2yz, + cubic group)
 *   A10/A11 all rates other than the shear rate equal to one
 *   A12 linear kinematic viscosity nu(phi)
 *   A13 n = grad(phi)/max(|grad(phi)|, 1e-4)
 *   A15 F_b = -(rho - (rho_h+rho_l)/2) g e_vertical
 *   A16 We = rho_h L U^2/sigma   A17 half-way bounce-back, mirrored phi ghosts
 *   A18 tanh initial profiles    A21 D2Q9 restriction of the 3-D relations
 *   A28 symmetry boundary of the 2-D splash (Sec. 3.4): half-way specular
 *       reflection -- a population leaving across the face of a symmetry
 *       axis returns to the same cell along that axis with its velocity
 *       component along the axis reversed (it still moves along the other
 *       axes); the phi ghost beyond the face equals the boundary cell
 * and, for the reduced phase lattice of Sec. 2.2 (LBMO_FLAG_PHASE_REDUCED):
 *   P1  D3Q7 (w 1/4 rest, 1/8 faces, cs2 = 1/4) / D2Q5 (1/3, 1/6, cs2 = 1/3)
 *   P2  d/dt(phi u) = (phi u)^n - (phi u)^(n-1); before the first step the
 *       previous value is the current one (init and set_state)
 *   P3  tau_bar_phi = M/cs2 + 1/2 with the phase lattice's cs2; C_bar takes
 *       the factor lambda of A4, like S_bar
 * and, with LBMO_FLAG_DIVU (the alternative to A6):
 *   V1  div(u) by the isotropic difference of the previous step's u (stored
 *       per cell; before the first step the current one), with the ghost
 *       velocity across a wall equal to minus the wall cell's (no slip)
 */
#include "lbmo.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CS2 (1.0 / 3.0)
#define KI(a, b, c) ((a) + 3 * (b) + 9 * (c))

static __thread char g_err[256];
static void set_err(const char *m) { snprintf(g_err, sizeof g_err, "%s", m); }
const char *lbmo_last_error(void) { return g_err; }

/* ------------------------------------------------------------------ lattice */
/* Velocities c in {-1,0,1}^D with Gauss-Hermite weights (Sec. 2.2): the D1Q3
 * weights 2/3 (rest) and 1/6 (moving), tensorised; c_s^2 = 1/3. */
typedef struct {
    int D, Q;
    int c[27][3];
    double w[27];
    double cs2;
} lattice;

static double w1(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }

static void lattice_build(int D, lattice *L)
{
    L->D = D;
    L->Q = (D == 3) ? 27 : 9;
    for (int a = 0; a < L->Q; ++a) {
        int cx = a % 3 - 1, cy = (a / 3) % 3 - 1, cz = (D == 3) ? a / 9 - 1 : 0;
        L->c[a][0] = cx;
        L->c[a][1] = cy;
        L->c[a][2] = cz;
        L->w[a] = w1(cx) * w1(cy) * (D == 3 ? w1(cz) : 1.0);
    }
    L->cs2 = CS2;
}

/* Lattice of the phase field.  The full lattice, or (reduced) its rest and
 * face directions in the same relative order, with the D3Q7 / D2Q5 weights
 * (reading P1): sum w = 1, sum w c = 0, sum w c c = cs2 I. */
static void phase_lattice_build(int D, int reduced, lattice *L)
{
    lattice full;
    lattice_build(D, &full);
    if (!reduced) {
        *L = full;
        return;
    }
    L->D = D;
    L->Q = 0;
    for (int a = 0; a < full.Q; ++a) {
        int moving = abs(full.c[a][0]) + abs(full.c[a][1]) + abs(full.c[a][2]);
        if (moving > 1) continue;
        for (int i = 0; i < 3; ++i) L->c[L->Q][i] = full.c[a][i];
        if (D == 3)
            L->w[L->Q] = moving ? 1.0 / 8.0 : 1.0 / 4.0;
        else
            L->w[L->Q] = moving ? 1.0 / 6.0 : 1.0 / 3.0;
        L->Q += 1;
    }
    L->cs2 = (D == 3) ? 0.25 : 1.0 / 3.0;
}

void lbmo_phase_lattice(int D, int reduced, int *Q, int *c, double *w, double *cs2)
{
    lattice L;
    phase_lattice_build(D, reduced, &L);
    *Q = L.Q;
    for (int a = 0; a < L.Q; ++a) {
        for (int i = 0; i < 3; ++i) c[3 * a + i] = L.c[a][i];
        w[a] = L.w[a];
    }
    *cs2 = L.cs2;
}

void lbmo_lattice(int D, int *Q, int *c, double *w)
{
    lattice L;
    lattice_build(D, &L);
    *Q = L.Q;
    for (int a = 0; a < L.Q; ++a) {
        for (int i = 0; i < 3; ++i) c[3 * a + i] = L.c[a][i];
        w[a] = L.w[a];
    }
}

/* ------------------------------------------------------------ the state */
struct lbmo {
    int D, Q, Qg, n[3], per[3], vert;
    long N;
    lattice L, Lg;      /* flow lattice, phase-field lattice */
    double *phiu_prev;  /* reduced phase lattice: phi u of the previous step, [3][cell] */
    double *u_prev, *u_next; /* LBMO_FLAG_DIVU: velocity of the previous / current step, [3][cell] */
    lbmo_phys phys;
    lbmo_derived d;
    double rate_shear, rate_bulk, r3, r4, r5, r6;
    double *f, *g, *fn, *gn, *phi;
    long step;
    int probe[3];
};

/* ------------------------------------------------------- parameter closure */
/* Derived lattice parameters from the problem statement:
 *   rho_h = 1 (Sec. 3 scales by the heavy density); At = (rho_h-rho_l)/(rho_h+rho_l)
 *   U_ref = U0 (splash, Sec. 3.4) or sqrt(g L_x) (Rayleigh-Taylor, Sec. 3.2)
 *   nu_h  = U_ref L / Re (Re = rho_h U L / mu_h)
 *   sigma = rho L U^2 / We (Sec. 3.4, reading A16)
 *   beta = 12 sigma / W, kappa = 3 sigma W / 2 (Sec. 2.1)
 *   tau_bar_phi = M / cs2 + 1/2 (Sec. 2.2), lambda = 1 - 1/(2 tau_bar_phi) (A4),
 *   cs2 of the phase-field lattice (P3) */
int lbmo_derive(int D, const lbmo_phys *p, lbmo_derived *o)
{
    const double cs2g = ((p->flags & LBMO_FLAG_PHASE_REDUCED) && D == 3) ? 0.25 : CS2;
    memset(o, 0, sizeof *o);
    o->rho_h = 1.0;
    if (p->atwood > 0.0) {
        if (p->atwood >= 1.0) { set_err("atwood must be < 1"); return -1; }
        o->rho_l = (1.0 - p->atwood) / (1.0 + p->atwood);
    } else {
        if (!(p->rho_ratio > 0.0)) { set_err("rho_ratio must be > 0"); return -1; }
        o->rho_l = 1.0 / p->rho_ratio;
    }
    if (p->U0 > 0.0)
        o->U_ref = p->U0;
    else
        o->U_ref = sqrt(fmax(p->g_accel, 0.0) * p->L_ref);
    if (p->nu_h > 0.0)
        o->nu_h = p->nu_h;
    else {
        if (!(p->Re > 0.0) || !(o->U_ref > 0.0) || !(p->L_ref > 0.0)) {
            set_err("need nu_h > 0 or Re, L_ref and a reference velocity");
            return -1;
        }
        o->nu_h = o->U_ref * p->L_ref / p->Re;
    }
    if (!(p->nu_ratio > 0.0)) { set_err("nu_ratio must be > 0"); return -1; }
    o->nu_l = o->nu_h * p->nu_ratio;
    if (p->sigma >= 0.0)
        o->sigma = p->sigma;
    else if (p->We > 0.0) {
        double rho_we = (p->flags & LBMO_FLAG_WE_LIGHT) ? o->rho_l : o->rho_h;
        o->sigma = rho_we * p->L_ref * o->U_ref * o->U_ref / p->We;
    } else
        o->sigma = 0.0;
    if (!(p->width > 0.0)) { set_err("width must be > 0"); return -1; }
    if (!(p->mobility > 0.0)) { set_err("mobility must be > 0"); return -1; }
    o->W = p->width;
    o->M = p->mobility;
    o->beta = 12.0 * o->sigma / o->W;
    o->kappa = 1.5 * o->sigma * o->W;
    o->tau_phi = o->M / cs2g + 0.5;
    o->lambda_phi = 1.0 - 1.0 / (2.0 * o->tau_phi);
    o->g_accel = p->g_accel;
    o->force_x = p->force_x;
    o->K_impact = (p->We > 0.0 && p->Re > 0.0) ? sqrt(p->We) * pow(p->Re, 0.25) : 0.0;
    return 0;
}

lbmo *lbmo_create(int D, const int dims[3], const int periodic[3], const lbmo_phys *p)
{
    if (D != 2 && D != 3) { set_err("D must be 2 or 3"); return NULL; }
    if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1 || (D == 2 && dims[2] != 1)) {
        set_err("bad dims");
        return NULL;
    }
    lbmo *s = (lbmo *)calloc(1, sizeof *s);
    if (!s) { set_err("out of memory"); return NULL; }
    s->D = D;
    lattice_build(D, &s->L);
    s->Q = s->L.Q;
    phase_lattice_build(D, (p->flags & LBMO_FLAG_PHASE_REDUCED) ? 1 : 0, &s->Lg);
    s->Qg = s->Lg.Q;
    for (int i = 0; i < 3; ++i) {
        s->n[i] = dims[i];
        s->per[i] = periodic[i] == 2 ? 2 : (periodic[i] ? 1 : 0);
    }
    if (D == 2) s->per[2] = 1;
    s->vert = (D == 3) ? 2 : 1;
    for (int i = 0; i < 3; ++i)
        if (s->per[i] == 2 && (i == s->vert || (p->flags & LBMO_FLAG_DIVU))) {
            set_err("a symmetry axis is horizontal and excludes the divergence term");
            free(s);
            return NULL;
        }
    s->N = (long)dims[0] * dims[1] * dims[2];
    s->phys = *p;
    if (lbmo_derive(D, p, &s->d) != 0) { free(s); return NULL; }
    s->rate_shear = -1.0;
    s->rate_bulk = s->r3 = s->r4 = s->r5 = s->r6 = 1.0;
    size_t bytes = sizeof(double) * (size_t)s->Q * (size_t)s->N;
    size_t gbytes = sizeof(double) * (size_t)s->Qg * (size_t)s->N;
    s->f = (double *)calloc(1, bytes);
    s->g = (double *)calloc(1, gbytes);
    s->fn = (double *)calloc(1, bytes);
    s->gn = (double *)calloc(1, gbytes);
    s->phi = (double *)calloc((size_t)s->N, sizeof(double));
    s->phiu_prev = (double *)calloc(3 * (size_t)s->N, sizeof(double));
    s->u_prev = (double *)calloc(3 * (size_t)s->N, sizeof(double));
    s->u_next = (double *)calloc(3 * (size_t)s->N, sizeof(double));
    if (!s->f || !s->g || !s->fn || !s->gn || !s->phi || !s->phiu_prev || !s->u_prev || !s->u_next) {
        lbmo_destroy(s);
        set_err("out of memory");
        return NULL;
    }
    for (int i = 0; i < 3; ++i) s->probe[i] = s->n[i] / 2;
    return s;
}

void lbmo_destroy(lbmo *s)
{
    if (!s) return;
    free(s->f);
    free(s->g);
    free(s->fn);
    free(s->gn);
    free(s->phi);
    free(s->phiu_prev);
    free(s->u_prev);
    free(s->u_next);
    free(s);
}

void lbmo_get_derived(const lbmo *s, lbmo_derived *out) { *out = s->d; }

void lbmo_set_rates(lbmo *s, double shear, double bulk, double r3, double r4, double r5, double r6)
{
    s->rate_shear = shear;
    s->rate_bulk = bulk;
    s->r3 = r3;
    s->r4 = r4;
    s->r5 = r5;
    s->r6 = r6;
}

void lbmo_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int lbmo_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------ indexing */
static long cell_index(const lbmo *s, int x, int y, int z) { return x + (long)s->n[0] * (y + (long)s->n[1] * z); }

/* neighbour coordinate for the phi stencil: periodic wrap, or the mirror image
 * across a half-way wall (reading A17: the ghost value equals the wall cell) */
static int ghost_coord(int x, int d, int n, int periodic)
{
    int y = x + d;
    if (y >= 0 && y < n) return y;
    if (periodic == 1) return ((y % n) + n) % n;
    return y < 0 ? 0 : n - 1; /* wall or symmetry face */
}

/* ------------------------------------------------ isotropic differences */
/* d_i phi = (1/cs2) sum_a w_a c_ai phi(x + c_a);
 * lap phi = (2/cs2) sum_a w_a [phi(x + c_a) - phi(x)]          (Sec. 2.2)
 * The gradient sum is grouped over opposite pairs, w_a c_ai [phi(x+c_a) -
 * phi(x-c_a)] for the half of the directions with a < opposite(a): the same
 * sum, but exactly zero on a uniform field, where a round-off gradient would
 * otherwise be blown up to a unit normal by the normalisation n = grad/|grad|. */
static void fd_cell(const lbmo *s, const double *field, int x, int y, int z, double grad[3], double *lap)
{
    const lattice *L = &s->L;
    double f0 = field[cell_index(s, x, y, z)];
    double gs[3] = {0.0, 0.0, 0.0}, ls = 0.0;
    for (int a = 0; a < L->Q; ++a) {
        int xx = ghost_coord(x, L->c[a][0], s->n[0], s->per[0]);
        int yy = ghost_coord(y, L->c[a][1], s->n[1], s->per[1]);
        int zz = ghost_coord(z, L->c[a][2], s->n[2], s->per[2]);
        double v = field[cell_index(s, xx, yy, zz)];
        ls += L->w[a] * (v - f0);
        if (a < L->Q - 1 - a) {
            int xm = ghost_coord(x, -L->c[a][0], s->n[0], s->per[0]);
            int ym = ghost_coord(y, -L->c[a][1], s->n[1], s->per[1]);
            int zm = ghost_coord(z, -L->c[a][2], s->n[2], s->per[2]);
            double vm = field[cell_index(s, xm, ym, zm)];
            for (int i = 0; i < 3; ++i) gs[i] += L->w[a] * L->c[a][i] * (v - vm);
        }
    }
    for (int i = 0; i < 3; ++i) grad[i] = gs[i] / CS2;
    *lap = 2.0 * ls / CS2;
}

/* div(u) at one cell (reading V1): (1/cs2) sum_a w_a c_a . u(x + c_a); a
 * neighbour across a wall is the mirror ghost of the wall cell with the
 * velocity reversed (no slip at the half-way wall) */
static double div_cell(const lbmo *s, const double *u, int x, int y, int z)
{
    const lattice *L = &s->L;
    const int xyz[3] = {x, y, z};
    double sum = 0.0;
    for (int a = 0; a < L->Q; ++a) {
        int q[3], sign = 1;
        for (int k = 0; k < 3; ++k) {
            int v = xyz[k] + L->c[a][k];
            if ((v < 0 || v >= s->n[k]) && s->per[k] == 0) sign = -1;
            q[k] = ghost_coord(xyz[k], L->c[a][k], s->n[k], s->per[k]);
        }
        long j = cell_index(s, q[0], q[1], q[2]);
        double cu = 0.0;
        for (int k = 0; k < 3; ++k) cu += L->c[a][k] * u[(size_t)k * s->N + j];
        sum += L->w[a] * sign * cu;
    }
    return sum / CS2;
}

void lbmo_divu(const lbmo *s, const double *u, double *div)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < s->N; ++i) {
        int x = (int)(i % s->n[0]), y = (int)((i / s->n[0]) % s->n[1]), z = (int)(i / ((long)s->n[0] * s->n[1]));
        div[i] = div_cell(s, u, x, y, z);
    }
}

void lbmo_fd(const lbmo *s, const double *field, double *grad, double *lap)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < s->N; ++i) {
        int x = (int)(i % s->n[0]), y = (int)((i / s->n[0]) % s->n[1]), z = (int)(i / ((long)s->n[0] * s->n[1]));
        double gr[3], l;
        fd_cell(s, field, x, y, z, gr, &l);
        for (int k = 0; k < 3; ++k) grad[3 * i + k] = gr[k];
        lap[i] = l;
    }
}

/* ---------------------------------------------- moments and cumulants */
static double ipow(double v, int k)
{
    double r = 1.0;
    for (int i = 0; i < k; ++i) r *= v;
    return r;
}

/* central moments  Pi_{x^a y^b z^c} = sum_al (cx-ux)^a (cy-uy)^b (cz-uz)^c h_al
 * by the direct definition (Sec. 2.3) */
void lbmo_central_moments(int D, const double *h, const double u[3], double *k)
{
    lattice L;
    lattice_build(D, &L);
    int cmax = (D == 3) ? 2 : 0;
    /* pw[i][p][c+1] = (c - u_i)^p, the factors of the definition */
    double pw[3][3][3];
    for (int i = 0; i < 3; ++i)
        for (int c = -1; c <= 1; ++c)
            for (int p = 0; p <= 2; ++p) pw[i][p][c + 1] = ipow(c - u[i], p);
    for (int i = 0; i < 27; ++i) k[i] = 0.0;
    for (int c = 0; c <= cmax; ++c)
        for (int b = 0; b <= 2; ++b)
            for (int a = 0; a <= 2; ++a) {
                double s = 0.0;
                for (int al = 0; al < L.Q; ++al)
                    s += pw[0][a][L.c[al][0] + 1] * pw[1][b][L.c[al][1] + 1] * pw[2][c][L.c[al][2] + 1] * h[al];
                k[KI(a, b, c)] = s;
            }
}

/* central moments -> cumulants for a normalised distribution (zeroth moment
 * one, first central moments zero), Sec. 2.3, with the corrections of reading
 * A9 for the sixth order; permutations written out. */
void lbmo_cumulants_forward(int D, const double *k, double *K)
{
    for (int i = 0; i < 27; ++i) K[i] = k[i];
    const double k200 = k[KI(2, 0, 0)], k020 = k[KI(0, 2, 0)], k002 = k[KI(0, 0, 2)];
    const double k110 = k[KI(1, 1, 0)], k101 = k[KI(1, 0, 1)], k011 = k[KI(0, 1, 1)];
    /* fourth order */
    K[KI(2, 2, 0)] = k[KI(2, 2, 0)] - (k200 * k020 + 2.0 * k110 * k110);
    if (D == 2) return;
    K[KI(2, 0, 2)] = k[KI(2, 0, 2)] - (k200 * k002 + 2.0 * k101 * k101);
    K[KI(0, 2, 2)] = k[KI(0, 2, 2)] - (k020 * k002 + 2.0 * k011 * k011);
    K[KI(2, 1, 1)] = k[KI(2, 1, 1)] - (k200 * k011 + 2.0 * k110 * k101);
    K[KI(1, 2, 1)] = k[KI(1, 2, 1)] - (k020 * k101 + 2.0 * k110 * k011);
    K[KI(1, 1, 2)] = k[KI(1, 1, 2)] - (k002 * k110 + 2.0 * k101 * k011);
    /* fifth order */
    const double k111 = k[KI(1, 1, 1)];
    const double k120 = k[KI(1, 2, 0)], k102 = k[KI(1, 0, 2)], k210 = k[KI(2, 1, 0)];
    const double k012 = k[KI(0, 1, 2)], k201 = k[KI(2, 0, 1)], k021 = k[KI(0, 2, 1)];
    K[KI(1, 2, 2)] = k[KI(1, 2, 2)] - (k002 * k120 + k020 * k102 + 4.0 * k011 * k111 + 2.0 * (k101 * k021 + k110 * k012));
    K[KI(2, 1, 2)] = k[KI(2, 1, 2)] - (k002 * k210 + k200 * k012 + 4.0 * k101 * k111 + 2.0 * (k011 * k201 + k110 * k102));
    K[KI(2, 2, 1)] = k[KI(2, 2, 1)] - (k020 * k201 + k200 * k021 + 4.0 * k110 * k111 + 2.0 * (k011 * k210 + k101 * k120));
    /* sixth order */
    const double k220 = k[KI(2, 2, 0)], k202 = k[KI(2, 0, 2)], k022 = k[KI(0, 2, 2)];
    const double k211 = k[KI(2, 1, 1)], k121 = k[KI(1, 2, 1)], k112 = k[KI(1, 1, 2)];
    double quad = 4.0 * k111 * k111 + k200 * k022 + k020 * k202 + k002 * k220 +
                  4.0 * (k011 * k211 + k101 * k121 + k110 * k112) + 2.0 * (k120 * k102 + k210 * k012 + k201 * k021);
    double cub = 16.0 * k110 * k101 * k011 + 4.0 * (k101 * k101 * k020 + k011 * k011 * k200 + k110 * k110 * k002) +
                 2.0 * k200 * k020 * k002;
    K[KI(2, 2, 2)] = k[KI(2, 2, 2)] - quad + cub;
}

/* cumulants -> central moments (inverse relations of Sec. 2.3, same reading) */
void lbmo_cumulants_inverse(int D, const double *K, double *k)
{
    for (int i = 0; i < 27; ++i) k[i] = K[i];
    const double k200 = k[KI(2, 0, 0)], k020 = k[KI(0, 2, 0)], k002 = k[KI(0, 0, 2)];
    const double k110 = k[KI(1, 1, 0)], k101 = k[KI(1, 0, 1)], k011 = k[KI(0, 1, 1)];
    k[KI(2, 2, 0)] = K[KI(2, 2, 0)] + (k200 * k020 + 2.0 * k110 * k110);
    if (D == 2) return;
    k[KI(2, 0, 2)] = K[KI(2, 0, 2)] + (k200 * k002 + 2.0 * k101 * k101);
    k[KI(0, 2, 2)] = K[KI(0, 2, 2)] + (k020 * k002 + 2.0 * k011 * k011);
    k[KI(2, 1, 1)] = K[KI(2, 1, 1)] + (k200 * k011 + 2.0 * k110 * k101);
    k[KI(1, 2, 1)] = K[KI(1, 2, 1)] + (k020 * k101 + 2.0 * k110 * k011);
    k[KI(1, 1, 2)] = K[KI(1, 1, 2)] + (k002 * k110 + 2.0 * k101 * k011);
    const double k111 = k[KI(1, 1, 1)];
    const double k120 = k[KI(1, 2, 0)], k102 = k[KI(1, 0, 2)], k210 = k[KI(2, 1, 0)];
    const double k012 = k[KI(0, 1, 2)], k201 = k[KI(2, 0, 1)], k021 = k[KI(0, 2, 1)];
    k[KI(1, 2, 2)] = K[KI(1, 2, 2)] + (k002 * k120 + k020 * k102 + 4.0 * k011 * k111 + 2.0 * (k101 * k021 + k110 * k012));
    k[KI(2, 1, 2)] = K[KI(2, 1, 2)] + (k002 * k210 + k200 * k012 + 4.0 * k101 * k111 + 2.0 * (k011 * k201 + k110 * k102));
    k[KI(2, 2, 1)] = K[KI(2, 2, 1)] + (k020 * k201 + k200 * k021 + 4.0 * k110 * k111 + 2.0 * (k011 * k210 + k101 * k120));
    const double k220 = k[KI(2, 2, 0)], k202 = k[KI(2, 0, 2)], k022 = k[KI(0, 2, 2)];
    const double k211 = k[KI(2, 1, 1)], k121 = k[KI(1, 2, 1)], k112 = k[KI(1, 1, 2)];
    double quad = 4.0 * k111 * k111 + k200 * k022 + k020 * k202 + k002 * k220 +
                  4.0 * (k011 * k211 + k101 * k121 + k110 * k112) + 2.0 * (k120 * k102 + k210 * k012 + k201 * k021);
    double cub = 16.0 * k110 * k101 * k011 + 4.0 * (k101 * k101 * k020 + k011 * k011 * k200 + k110 * k110 * k002) +
                 2.0 * k200 * k020 * k002;
    k[KI(2, 2, 2)] = K[KI(2, 2, 2)] + quad - cub;
}

/* central moments about u -> populations.  Per axis (the moment map is a
 * tensor product): raw m0 = k0, m1 = k1 + u k0, m2 = k2 + 2u k1 + u^2 k0, then
 * f(0) = m0 - m2, f(+-1) = (m2 +- m1)/2. */
static void axis_inverse(double k0, double k1, double k2, double u, double out[3])
{
    double m0 = k0, m1 = k1 + u * k0, m2 = k2 + 2.0 * u * k1 + u * u * k0;
    out[0] = 0.5 * (m2 - m1); /* c = -1 */
    out[1] = m0 - m2;         /* c =  0 */
    out[2] = 0.5 * (m2 + m1); /* c = +1 */
}

void lbmo_kron_inverse(int D, const double *k, const double u[3], double *h)
{
    double A[27], B[27], out[3];
    int cmax = (D == 3) ? 2 : 0;
    /* x: (a,b,c) -> (cx,b,c) */
    for (int c = 0; c <= cmax; ++c)
        for (int b = 0; b <= 2; ++b) {
            axis_inverse(k[KI(0, b, c)], k[KI(1, b, c)], k[KI(2, b, c)], u[0], out);
            for (int i = 0; i < 3; ++i) A[KI(i, b, c)] = out[i];
        }
    /* y: (cx,b,c) -> (cx,cy,c) */
    for (int c = 0; c <= cmax; ++c)
        for (int i = 0; i < 3; ++i) {
            axis_inverse(A[KI(i, 0, c)], A[KI(i, 1, c)], A[KI(i, 2, c)], u[1], out);
            for (int j = 0; j < 3; ++j) B[KI(i, j, c)] = out[j];
        }
    if (D == 2) {
        for (int j = 0; j < 3; ++j)
            for (int i = 0; i < 3; ++i) h[i + 3 * j] = B[KI(i, j, 0)];
        return;
    }
    /* z: (cx,cy,c) -> (cx,cy,cz) */
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
            axis_inverse(B[KI(i, j, 0)], B[KI(i, j, 1)], B[KI(i, j, 2)], u[2], out);
            for (int l = 0; l < 3; ++l) h[KI(i, j, l)] = out[l];
        }
}

/* relaxation in cumulant space (Sec. 2.3): shear rate on the off-diagonal and
 * deviatoric second-order cumulants, bulk rate on the trace (equilibrium
 * D cs2), order-n rates on every higher cumulant (equilibrium 0). */
static void relax(const lbmo *s, int D, double *K, double om)
{
    double ob = s->rate_bulk;
    K[KI(1, 1, 0)] *= (1.0 - om);
    if (D == 3) {
        K[KI(1, 0, 1)] *= (1.0 - om);
        K[KI(0, 1, 1)] *= (1.0 - om);
        double kxx = K[KI(2, 0, 0)], kyy = K[KI(0, 2, 0)], kzz = K[KI(0, 0, 2)];
        double d1 = (1.0 - om) * (kxx - kyy), d2 = (1.0 - om) * (kxx - kzz);
        double T = kxx + kyy + kzz;
        T -= ob * (T - 3.0 * CS2);
        K[KI(2, 0, 0)] = (T + d1 + d2) / 3.0;
        K[KI(0, 2, 0)] = (T - 2.0 * d1 + d2) / 3.0;
        K[KI(0, 0, 2)] = (T + d1 - 2.0 * d2) / 3.0;
    } else {
        double kxx = K[KI(2, 0, 0)], kyy = K[KI(0, 2, 0)];
        double d1 = (1.0 - om) * (kxx - kyy);
        double T = kxx + kyy;
        T -= ob * (T - 2.0 * CS2);
        K[KI(2, 0, 0)] = 0.5 * (T + d1);
        K[KI(0, 2, 0)] = 0.5 * (T - d1);
    }
    const double rate[7] = {0, 0, 0, s->r3, s->r4, s->r5, s->r6};
    int cmax = (D == 3) ? 2 : 0;
    for (int c = 0; c <= cmax; ++c)
        for (int b = 0; b <= 2; ++b)
            for (int a = 0; a <= 2; ++a) {
                int order = a + b + c;
                if (order >= 3) K[KI(a, b, c)] *= (1.0 - rate[order]);
            }
}

/* ---------------------------------------------------- local closure */
typedef struct {
    double rho, nu, omega, n[3], mu, F[3], u[3], P, gradrho[3];
} closure;

/* rho(phi) (Sec. 2.3), nu(phi) (A12), omega (A7), n (A13), mu_phi (A1),
 * F = mu grad(phi) + F_b (A2, A15), and u = J/(rho cs2) + F/(2 rho), the
 * velocity for which the pre-conditioned populations have first moment u. */
static void local_closure(const lbmo *s, const double *f, double phi, const double grad[3], double lap, closure *c)
{
    const lattice *L = &s->L;
    const lbmo_derived *d = &s->d;
    double drho = d->rho_h - d->rho_l;
    c->rho = d->rho_l + drho * phi;
    if (s->phys.flags & LBMO_FLAG_DYNAMIC_VISC) {
        double eta = d->rho_l * d->nu_l + (d->rho_h * d->nu_h - d->rho_l * d->nu_l) * phi;
        c->nu = eta / c->rho;
    } else
        c->nu = d->nu_h + (d->nu_l - d->nu_h) * (1.0 - phi);
    c->omega = (s->rate_shear > 0.0) ? s->rate_shear : 1.0 / (c->nu / CS2 + 0.5);
    double gn = sqrt(grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]);
    double den = fmax(gn, 1e-4);
    for (int i = 0; i < 3; ++i) c->n[i] = grad[i] / den;
    c->mu = 2.0 * d->beta * phi * (phi - 1.0) * (2.0 * phi - 1.0) - d->kappa * lap;
    for (int i = 0; i < 3; ++i) c->F[i] = c->mu * grad[i];
    if (s->phys.flags & LBMO_FLAG_UNIFORM_FORCE)
        c->F[0] += d->force_x;
    else
        c->F[s->vert] -= (c->rho - 0.5 * (d->rho_h + d->rho_l)) * d->g_accel;
    double P = 0.0, J[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < L->Q; ++a) {
        P += f[a];
        for (int i = 0; i < 3; ++i) J[i] += L->c[a][i] * f[a];
    }
    c->P = P;
    for (int i = 0; i < 3; ++i) {
        c->u[i] = J[i] / (c->rho * CS2) + c->F[i] / (2.0 * c->rho);
        c->gradrho[i] = drho * grad[i];
    }
}

/* normalised second-order Hermite equilibrium f_eq/rho (App. A):
 * w [1 + c.u/cs2 + ((c.u)^2 - cs2 u^2)/(2 cs4)] */
static double gamma_eq(const lattice *L, int a, const double u[3])
{
    double cu = L->c[a][0] * u[0] + L->c[a][1] * u[1] + L->c[a][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return L->w[a] * (1.0 + cu / CS2 + (cu * cu - CS2 * uu) / (2.0 * CS2 * CS2));
}

void lbmo_collide_cell(const lbmo *s, const double *f, const double *g, double phi, const double grad[3], double lap,
                       double *fout, double *gout, double *diag)
{
    lbmo_collide_cell_prev(s, f, g, phi, grad, lap, NULL, fout, gout, diag);
}

int lbmo_phase_q(const lbmo *s) { return s->Qg; }

void lbmo_collide_cell_prev(const lbmo *s, const double *f, const double *g, double phi, const double grad[3],
                            double lap, const double *phiu_prev, double *fout, double *gout, double *diag)
{
    lbmo_collide_cell_ex(s, f, g, phi, grad, lap, phiu_prev, 0.0, fout, gout, diag);
}

void lbmo_collide_cell_ex(const lbmo *s, const double *f, const double *g, double phi, const double grad[3],
                          double lap, const double *phiu_prev, double divu, double *fout, double *gout, double *diag)
{
    const lattice *L = &s->L;
    const lbmo_derived *d = &s->d;
    const int Q = L->Q, D = L->D;
    closure c;
    local_closure(s, f, phi, grad, lap, &c);
    const double *u = c.u;

    /* source Xi (Sec. 2.3, reading A6) */
    double Xi[27], sumXi = 0.0, sumcXi[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < Q; ++a) {
        double G = gamma_eq(L, a, u);
        double cmu_grho = 0.0, cmu_F = 0.0;
        for (int i = 0; i < 3; ++i) {
            cmu_grho += (L->c[a][i] - u[i]) * c.gradrho[i];
            cmu_F += (L->c[a][i] - u[i]) * c.F[i];
        }
        Xi[a] = CS2 * (G - L->w[a]) * cmu_grho + cmu_F * G;
        if (s->phys.flags & LBMO_FLAG_DIVU) Xi[a] += L->w[a] * CS2 * c.rho * divu; /* w cs2 rho div(u), V1 */
        sumXi += Xi[a];
        for (int i = 0; i < 3; ++i) sumcXi[i] += L->c[a][i] * Xi[a];
    }
    /* pre-conditioning f^p = f'/(rho cs2) + Xi/(2 rho cs2) */
    double fp[27], h[27], theta = 0.0;
    for (int a = 0; a < Q; ++a) {
        fp[a] = f[a] / (c.rho * CS2) + Xi[a] / (2.0 * c.rho * CS2);
        theta += fp[a];
    }
    /* A8: collide h = f^p - w (theta - 1), sum h = 1 */
    for (int a = 0; a < Q; ++a) h[a] = fp[a] - L->w[a] * (theta - 1.0);
    double kap[27], K[27], kstar[27], hs[27];
    lbmo_central_moments(D, h, u, kap);
    lbmo_cumulants_forward(D, kap, K);
    relax(s, D, K, c.omega);
    lbmo_cumulants_inverse(D, K, kstar);
    lbmo_kron_inverse(D, kstar, u, hs);
    /* f'* = rho cs2 f^p* + Xi/2, f^p* = h* + w (theta - 1) */
    for (int a = 0; a < Q; ++a) fout[a] = c.rho * CS2 * (hs[a] + L->w[a] * (theta - 1.0)) + 0.5 * Xi[a];

    /* phase field: BGK towards g_eq with the sharpening source (Sec. 2.2) */
    const lattice *Lg = &s->Lg;
    const int reduced = (s->phys.flags & LBMO_FLAG_PHASE_REDUCED) != 0;
    double X = 4.0 * phi * (1.0 - phi) / d->W;
    double phiu[3], dphiu[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 3; ++i) {
        phiu[i] = phi * u[i];
        if (reduced && phiu_prev) dphiu[i] = phiu[i] - phiu_prev[i]; /* d/dt(phi u), reading P2 */
    }
    for (int a = 0; a < Lg->Q; ++a) {
        double cn = Lg->c[a][0] * c.n[0] + Lg->c[a][1] * c.n[1] + Lg->c[a][2] * c.n[2];
        double geq, corr = 0.0;
        if (reduced) {
            /* first-order equilibrium w phi (1 + c.u/cs2) and the correction
             * C_bar = lambda (w/cs2) c . d/dt(phi u) (Sec. 2.2) */
            double cu = Lg->c[a][0] * u[0] + Lg->c[a][1] * u[1] + Lg->c[a][2] * u[2];
            double cd = Lg->c[a][0] * dphiu[0] + Lg->c[a][1] * dphiu[1] + Lg->c[a][2] * dphiu[2];
            geq = Lg->w[a] * phi * (1.0 + cu / Lg->cs2);
            corr = d->lambda_phi * Lg->w[a] * cd / Lg->cs2;
        } else {
            geq = phi * gamma_eq(L, a, u);
        }
        gout[a] = g[a] - (g[a] - geq) / d->tau_phi + d->lambda_phi * Lg->w[a] * cn * X + corr;
    }
    if (diag) {
        diag[0] = c.rho;
        for (int i = 0; i < 3; ++i) diag[1 + i] = u[i];
        diag[4] = c.P + 0.5 * sumXi;
        diag[5] = theta;
        diag[6] = c.omega;
        for (int i = 0; i < 3; ++i) diag[7 + i] = c.F[i];
        diag[10] = sumXi;
        for (int i = 0; i < 3; ++i) diag[11 + i] = sumcXi[i];
        for (int i = 0; i < 3; ++i) diag[14 + i] = phiu[i];
    }
}

/* ------------------------------------------------------------- stepping */
static void update_phi(lbmo *s)
{
    const int Q = s->Qg;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < s->N; ++i) {
        double p = 0.0;
        for (int a = 0; a < Q; ++a) p += s->g[(size_t)a * s->N + i];
        s->phi[i] = p; /* phi = sum_a g_a (Sec. 2.2) */
    }
}

/* direction of the lattice whose velocity is that of a with the components
 * flagged in flip reversed */
static int mirror_dir(const lattice *L, int a, const int flip[3])
{
    for (int b = 0; b < L->Q; ++b) {
        int same = 1;
        for (int k = 0; k < 3; ++k) same &= L->c[b][k] == (flip[k] ? -L->c[a][k] : L->c[a][k]);
        if (same) return b;
    }
    return a;
}

/* push population value v of direction a of the cell at xyz into the array
 * set out (lattice Lx): to the downstream cell; back into the same cell in
 * the opposite direction across a half-way wall (A17); across the face of a
 * symmetry axis, into the cell that is downstream along the other axes only,
 * with the velocity component along the symmetry axis reversed (A28).  A
 * link that crosses a wall bounces back whatever else it crosses. */
static void push(const lbmo *s, const lattice *Lx, double *out, int a, const int xyz[3], long i, double v)
{
    const int *c = Lx->c[a];
    int dst[3], wall = 0, flip[3] = {0, 0, 0}, mirrored = 0;
    for (int k = 0; k < 3; ++k) {
        int p = xyz[k] + c[k];
        if (p < 0 || p >= s->n[k]) {
            if (s->per[k] == 1) {
                p = (p + s->n[k]) % s->n[k];
            } else if (s->per[k] == 2) {
                p = xyz[k];
                flip[k] = mirrored = 1;
            } else {
                wall = 1;
            }
        }
        dst[k] = p;
    }
    if (wall) {
        out[(size_t)(Lx->Q - 1 - a) * s->N + i] = v;
    } else {
        const int b = mirrored ? mirror_dir(Lx, a, flip) : a;
        out[(size_t)b * s->N + cell_index(s, dst[0], dst[1], dst[2])] = v;
    }
}

static void step_once(lbmo *s)
{
    const lattice *L = &s->L, *Lg = &s->Lg;
    const int Q = s->Q, Qg = s->Qg;
    const long N = s->N;
    const int reduced = (s->phys.flags & LBMO_FLAG_PHASE_REDUCED) != 0;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        int x = (int)(i % s->n[0]), y = (int)((i / s->n[0]) % s->n[1]), z = (int)(i / ((long)s->n[0] * s->n[1]));
        double fl[27], gl[27], fo[27], go[27], grad[3], lap, diag[17], prev[3];
        for (int a = 0; a < Q; ++a) fl[a] = s->f[(size_t)a * N + i];
        for (int a = 0; a < Qg; ++a) gl[a] = s->g[(size_t)a * N + i];
        for (int k = 0; k < 3; ++k) prev[k] = s->phiu_prev[(size_t)k * N + i];
        fd_cell(s, s->phi, x, y, z, grad, &lap);
        const double divu = (s->phys.flags & LBMO_FLAG_DIVU) ? div_cell(s, s->u_prev, x, y, z) : 0.0;
        lbmo_collide_cell_ex(s, fl, gl, s->phi[i], grad, lap, reduced ? prev : NULL, divu, fo, go, diag);
        /* this step's phi u becomes the previous value of the next step (P2);
         * each cell reads and writes only its own entry */
        for (int k = 0; k < 3; ++k) s->phiu_prev[(size_t)k * N + i] = diag[14 + k];
        /* this step's u, read by the neighbours' div(u) of the next step (V1) */
        for (int k = 0; k < 3; ++k) s->u_next[(size_t)k * N + i] = diag[1 + k];
        /* push streaming; half-way bounce-back at walls */
        int xyz[3] = {x, y, z};
        for (int a = 0; a < Q; ++a) push(s, L, s->fn, a, xyz, i, fo[a]);
        for (int a = 0; a < Qg; ++a) push(s, Lg, s->gn, a, xyz, i, go[a]);
    }
    double *t = s->f;
    s->f = s->fn;
    s->fn = t;
    t = s->u_prev;
    s->u_prev = s->u_next;
    s->u_next = t;
    t = s->g;
    s->g = s->gn;
    s->gn = t;
    update_phi(s);
    s->step += 1;
}

void lbmo_step(lbmo *s, long n)
{
    for (long k = 0; k < n; ++k) step_once(s);
}

void lbmo_get_state(const lbmo *s, double *f, double *g, double *phi)
{
    size_t bytes = sizeof(double) * (size_t)s->Q * (size_t)s->N;
    size_t gbytes = sizeof(double) * (size_t)s->Qg * (size_t)s->N;
    if (f) memcpy(f, s->f, bytes);
    if (g) memcpy(g, s->g, gbytes);
    if (phi) memcpy(phi, s->phi, sizeof(double) * (size_t)s->N);
}

/* phi u of every cell from the current state (the u the next step's closure
 * computes): the previous value before the first step (reading P2) */
static void reset_phiu(lbmo *s)
{
    const long N = s->N;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        int x = (int)(i % s->n[0]), y = (int)((i / s->n[0]) % s->n[1]), z = (int)(i / ((long)s->n[0] * s->n[1]));
        double fl[27], grad[3], lap;
        for (int a = 0; a < s->Q; ++a) fl[a] = s->f[(size_t)a * N + i];
        fd_cell(s, s->phi, x, y, z, grad, &lap);
        closure c;
        local_closure(s, fl, s->phi[i], grad, lap, &c);
        for (int k = 0; k < 3; ++k) {
            s->phiu_prev[(size_t)k * N + i] = s->phi[i] * c.u[k];
            s->u_prev[(size_t)k * N + i] = c.u[k]; /* V1: the previous u before the first step */
        }
    }
}

void lbmo_set_state(lbmo *s, const double *f, const double *g)
{
    size_t bytes = sizeof(double) * (size_t)s->Q * (size_t)s->N;
    size_t gbytes = sizeof(double) * (size_t)s->Qg * (size_t)s->N;
    memcpy(s->f, f, bytes);
    memcpy(s->g, g, gbytes);
    update_phi(s);
    reset_phiu(s);
}

/* --------------------------------------------------------- initial state */
/* splitmix64 (Steele, Lea & Flood 2014): the output of the (counter+1)-th call
 * of a generator whose state starts at seed. */
unsigned long long lbmo_splitmix64(unsigned long long seed, unsigned long long counter)
{
    unsigned long long z = seed + (counter + 1ULL) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static double uniform01(unsigned long long seed, unsigned long long counter)
{
    return (double)(lbmo_splitmix64(seed, counter) >> 11) * (1.0 / 9007199254740992.0);
}

static double tanh_profile(double dist, double W) { return 0.5 * (1.0 + tanh(2.0 * dist / W)); }

int lbmo_init(lbmo *s, int case_id, const double *args, int nargs, unsigned long long seed)
{
    const lattice *L = &s->L, *Lg = &s->Lg;
    const int reduced = (s->phys.flags & LBMO_FLAG_PHASE_REDUCED) != 0;
    const lbmo_derived *d = &s->d;
    const int D = s->D, Q = s->Q, v = s->vert;
    const long N = s->N;
    const double PI = 3.14159265358979323846;
    double A[8] = {0};
    for (int i = 0; i < nargs && i < 8; ++i) A[i] = args[i];
    int need[7] = {3, 3, 3, 1, 4, 2, 5};
    if (case_id < 0 || case_id > 6) { set_err("unknown case"); return -1; }
    if (nargs < need[case_id]) { set_err("too few case arguments"); return -1; }
    double noise = 0.0;
    switch (case_id) {
    case LBMO_CASE_RT: noise = A[2]; break;
    case LBMO_CASE_DROP_STATIC: noise = A[2]; break;
    case LBMO_CASE_FLAT: noise = A[2]; break;
    case LBMO_CASE_POISEUILLE: noise = A[0]; break;
    case LBMO_CASE_DROP_SHEET: noise = A[3]; break;
    case LBMO_CASE_SHEAR_WAVE: noise = A[1]; break;
    default: noise = 0.0;
    }
    for (int i = 0; i < 3; ++i) s->probe[i] = s->n[i] / 2;
    if (D == 2) s->probe[2] = 0;
    if (case_id == LBMO_CASE_DROP_SHEET) {
        double zc = A[1] + 0.5 * A[0] + 2.0 * d->W;
        s->probe[v] = (int)floor(zc + 0.5);
    }
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        int x = (int)(i % s->n[0]), y = (int)((i / s->n[0]) % s->n[1]), z = (int)(i / ((long)s->n[0] * s->n[1]));
        double pos[3] = {(double)x, (double)y, (double)z};
        double hv = pos[v]; /* vertical coordinate */
        double phi = 0.0, p = 0.0, u[3] = {0.0, 0.0, 0.0};
        switch (case_id) {
        case LBMO_CASE_RT: {
            /* heavy above h(x,y) = h0 + amp [cos(2 pi x/nx) + cos(2 pi y/ny)] (Sec. 3.2/3.3) */
            double h = A[0] + A[1] * cos(2.0 * PI * x / s->n[0]);
            if (D == 3) h += A[1] * cos(2.0 * PI * y / s->n[1]);
            phi = tanh_profile(hv - h, d->W);
            /* optional hydrostatic start: dp/dz = -(rho - rho_bar) g along each column,
             * i.e. p = -g (rho_h - rho_l) (W/4) ln cosh(2 (z - h)/W), zero at the interface */
            if (nargs > 3 && A[3] != 0.0) {
                double t = 2.0 * (hv - h) / d->W, at = fabs(t);
                double lncosh = at + log1p(exp(-2.0 * at)) - log(2.0);
                p = -d->g_accel * (d->rho_h - d->rho_l) * 0.25 * d->W * lncosh;
            }
            break;
        }
        case LBMO_CASE_DROP_STATIC: {
            double r2 = 0.0;
            for (int k = 0; k < D; ++k) {
                double dx = pos[k] - s->n[k] / 2;
                r2 += dx * dx;
            }
            phi = tanh_profile(A[0] - sqrt(r2), d->W);
            if (A[1] != 0.0) p = (D == 3 ? 2.0 : 1.0) * d->sigma / A[0] * phi;
            break;
        }
        case LBMO_CASE_FLAT: {
            double dist = fmin(pos[0] - A[0], A[1] - pos[0]);
            phi = tanh_profile(dist, d->W);
            break;
        }
        case LBMO_CASE_POISEUILLE: {
            double vc = 0.5 * (s->n[v] - 1);
            phi = tanh_profile(vc - hv, d->W);
            break;
        }
        case LBMO_CASE_DROP_SHEET: {
            double Dd = A[0], sheet = A[1], U0 = A[2];
            double zc = sheet + 0.5 * Dd + 2.0 * d->W;
            double r2 = 0.0;
            for (int k = 0; k < D; ++k) {
                /* the drop's axis: at n/2, or at the coordinate given (on a
                 * symmetry face, -0.5, for a half domain) */
                double c0 = (k == v) ? zc : (nargs > 4 ? A[4] : (double)(s->n[k] / 2));
                double dx = pos[k] - c0;
                r2 += dx * dx;
            }
            double d_drop = 0.5 * Dd - sqrt(r2);
            double d_sheet = sheet - hv;
            phi = tanh_profile(fmax(d_drop, d_sheet), d->W);
            u[v] = -U0 * tanh_profile(d_drop, d->W);
            break;
        }
        case LBMO_CASE_SHEAR_WAVE:
            phi = 1.0;
            u[0] = A[0] * sin(2.0 * PI * y / s->n[1]);
            break;
        case LBMO_CASE_UNIFORM:
            phi = A[0];
            p = A[1];
            u[0] = A[2];
            u[1] = A[3];
            u[2] = (D == 3) ? A[4] : 0.0;
            break;
        }
        if (noise != 0.0) {
            for (int k = 0; k < D; ++k)
                u[k] += noise * d->U_ref * (2.0 * uniform01(seed, 3ULL * (unsigned long long)i + k) - 1.0) * phi;
        }
        double rho = d->rho_l + (d->rho_h - d->rho_l) * phi;
        for (int a = 0; a < Q; ++a) {
            double G = gamma_eq(L, a, u);
            /* f'_eq = w p_h + rho cs2 (Gamma - w)   (Sec. 2.3, App. A) */
            s->f[(size_t)a * N + i] = L->w[a] * p + rho * CS2 * (G - L->w[a]);
            if (!reduced) s->g[(size_t)a * N + i] = phi * G;
        }
        if (reduced) {
            /* first-order phase-field equilibrium (Sec. 2.2) */
            for (int a = 0; a < Lg->Q; ++a) {
                double cu = Lg->c[a][0] * u[0] + Lg->c[a][1] * u[1] + Lg->c[a][2] * u[2];
                s->g[(size_t)a * N + i] = Lg->w[a] * phi * (1.0 + cu / Lg->cs2);
            }
        }
    }
    update_phi(s);
    reset_phiu(s);
    s->step = 0;
    return 0;
}

/* ------------------------------------------------------------ observables */
typedef struct {
    double rho, p, u[3];
} macro;

static void cell_macro(const lbmo *s, long i, macro *m)
{
    const int Q = s->Q;
    int x = (int)(i % s->n[0]), y = (int)((i / s->n[0]) % s->n[1]), z = (int)(i / ((long)s->n[0] * s->n[1]));
    double fl[27], grad[3], lap;
    for (int a = 0; a < Q; ++a) fl[a] = s->f[(size_t)a * s->N + i];
    fd_cell(s, s->phi, x, y, z, grad, &lap);
    closure c;
    local_closure(s, fl, s->phi[i], grad, lap, &c);
    m->rho = c.rho;
    /* p_h = P + sum(Xi)/2 with sum(Xi) = cs2 u . grad(rho) (+ cs2 rho div(u) of
     * the stored previous u with LBMO_FLAG_DIVU: what the next step uses) */
    double ug = c.u[0] * c.gradrho[0] + c.u[1] * c.gradrho[1] + c.u[2] * c.gradrho[2];
    m->p = c.P + 0.5 * CS2 * ug;
    if (s->phys.flags & LBMO_FLAG_DIVU) m->p += 0.5 * CS2 * c.rho * div_cell(s, s->u_prev, x, y, z);
    for (int k = 0; k < 3; ++k) m->u[k] = c.u[k];
}

void lbmo_fields(const lbmo *s, double *rho, double *p, double *u)
{
#pragma omp parallel for schedule(static)
    for (long i = 0; i < s->N; ++i) {
        macro m;
        cell_macro(s, i, &m);
        if (rho) rho[i] = m.rho;
        if (p) p[i] = m.p;
        if (u)
            for (int k = 0; k < s->D; ++k) u[(size_t)k * s->N + i] = m.u[k];
    }
}

static double block_pressure(const lbmo *s, const int c0[3])
{
    double sum = 0.0;
    int cnt = 0;
    int r2 = (s->D == 3) ? 1 : 0;
    for (int dz = -r2; dz <= r2; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int x = ghost_coord(c0[0], dx, s->n[0], s->per[0]);
                int y = ghost_coord(c0[1], dy, s->n[1], s->per[1]);
                int z = ghost_coord(c0[2], dz, s->n[2], s->per[2]);
                macro m;
                cell_macro(s, cell_index(s, x, y, z), &m);
                sum += m.p;
                cnt += 1;
            }
    return sum / cnt;
}

static double column_phi(const lbmo *s, int hx, int hy, int k)
{
    int c[3] = {hx, hy, 0};
    if (s->D == 2) c[1] = k;
    else c[2] = k;
    return s->phi[cell_index(s, c[0], c[1], c[2])];
}

void lbmo_observables(const lbmo *s, lbmo_obs *o)
{
    memset(o, 0, sizeof *o);
    const long N = s->N;
    double mass = 0.0, ke = 0.0, umax = 0.0;
    int bad = 0;
    for (long i = 0; i < N; ++i) mass += s->phi[i];
    double *ke_c = (double *)malloc(sizeof(double) * (size_t)N);
    double *um_c = (double *)malloc(sizeof(double) * (size_t)N);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        macro m;
        cell_macro(s, i, &m);
        double uu = m.u[0] * m.u[0] + m.u[1] * m.u[1] + m.u[2] * m.u[2];
        ke_c[i] = 0.5 * m.rho * uu;
        um_c[i] = sqrt(uu);
    }
    for (long i = 0; i < N; ++i) {
        ke += ke_c[i];
        if (!(um_c[i] <= umax)) umax = um_c[i]; /* NaN propagates */
        if (!isfinite(ke_c[i]) || !isfinite(s->phi[i])) bad = 1;
    }
    free(ke_c);
    free(um_c);
    o->mass = mass;
    o->kinetic_energy = ke;
    o->max_u = umax;
    int corner[3] = {0, 0, 0};
    o->p_in = block_pressure(s, s->probe);
    o->p_out = block_pressure(s, corner);
    o->laplace_dp = o->p_in - o->p_out;
    /* phi = 1/2 crossings along the spike column (centre) and bubble column (origin) */
    int nv = s->n[s->vert];
    int sx = s->n[0] / 2, sy = (s->D == 3) ? s->n[1] / 2 : 0;
    o->tip_spike = -1.0;
    for (int k = 0; k < nv; ++k) {
        double pk = column_phi(s, sx, sy, k);
        if (pk >= 0.5) {
            if (k == 0) o->tip_spike = 0.0;
            else {
                double pm = column_phi(s, sx, sy, k - 1);
                o->tip_spike = k - (pk - 0.5) / (pk - pm);
            }
            break;
        }
    }
    o->tip_bubble = -1.0;
    for (int k = nv - 1; k >= 0; --k) {
        double pk = column_phi(s, 0, 0, k);
        if (pk < 0.5) {
            if (k == nv - 1) o->tip_bubble = (double)k;
            else {
                double pp = column_phi(s, 0, 0, k + 1);
                o->tip_bubble = k + (0.5 - pk) / (pp - pk);
            }
            break;
        }
    }
    o->step = s->step;
    o->health = bad ? 1 : 0;
}
