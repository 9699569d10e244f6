// lbmp_kernels.cu -- the reference step pair (phi pass + one thread per cell),
// initial conditions, state conversion and the FP64 observables.
//
// Streaming is "pull" with two population sets: step t reads set t&1 at the
// upstream cell x - c_a and writes its post-collision values to set 1-(t&1)
// at x.  Across a half-way bounce-back wall the upstream value is the
// opposite population of the cell itself (Sec. 3.2 boundary treatment).
#include <math.h>

#include "lbmp_internal.h"

namespace lbmp {

// ------------------------------------------------------------- phi pass
// value of the post-streaming population a of cell (x,y,z)
template <int D, class St>
__device__ __forceinline__ float pulled_value(const DevParams& p, const Pop<D, St>& set, int a, int x, int y, int z,
                                              long long i)
{
    int dir;
    const long long c = pull_src<D>(p, a, x, y, z, i, dir);
    return set.load(dir, c);
}

template <int D, class St, bool PR>
__global__ void phi_pass_kernel(DevParams p, Pop<D, St> g, float* __restrict__ phi)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int x, y, z;
    cell_xyz(p, i, x, y, z);
    float hi, lo;
    if constexpr (St::shifted) {
        phi_sum_shifted<D>(
            [&](int a, float& wr, float& wq) {
                int dir;
                const long long c = pull_src<D>(p, a, x, y, z, i, dir);
                g.load_parts(dir, c, wr, wq);
            },
            hi, lo);
    } else {
        phi_sum_phase<D, PR>(
            [&](int r) {
                int slot;
                const long long c = pull_src_g<D, PR>(p, r, x, y, z, i, slot);
                return g.load(slot, c);
            },
            hi, lo);
    }
    phi[i] = hi;  // phi = sum_a g_a (Sec. 2.2), as hi + lo
    phi[p.N + i] = lo;
}

// ----------------------------------------------------- reference step
// kFlagDivU: div(u) = (1/cs2) sum_a w_a c_a . u(x + c_a) of the stored
// previous velocity us ([k][cell], k < D); a neighbour across a wall is the
// wall cell's mirror ghost with the velocity reversed (no slip)
template <int D>
__device__ __forceinline__ float div_stored(const DevParams& p, const float* __restrict__ us, int x, int y, int z)
{
    constexpr int Q = Lat<D>::Q;
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int cx = Lat<D>::cx(a), cy = Lat<D>::cy(a), cz = Lat<D>::cz(a);
        const int xx = wrap_h(x + cx, p.nx);
        long long j;
        bool across;
        if (D == 3) {
            const int zr = z + cz;
            across = !p.vert_periodic && (zr < 0 || zr >= p.nz);
            j = ((long long)wrap_v(zr, p.nz, p.vert_periodic) * p.ny + wrap_h(y + cy, p.ny)) * p.nx + xx;
        } else {
            const int yr = y + cy;
            across = !p.vert_periodic && (yr < 0 || yr >= p.ny);
            j = (long long)wrap_v(yr, p.ny, p.vert_periodic) * p.nx + xx;
        }
        float cu = cx * us[j] + cy * us[p.N + j];
        if (D == 3) cu += cz * us[2 * p.N + j];
        acc += Lat<D>::w(a) * (across ? -cu : cu);
    }
    return 3.0f * acc;
}

// phiu (reduced phase lattice): phi u of the previous step per cell, [k][cell],
// read and replaced by this step's value (each cell touches only its own)
// us_in / us_out (kFlagDivU): the stored velocity of the previous step, read
// at the neighbours for div(u), and this step's, written per cell
template <int D, class St, bool PR>
__global__ void __launch_bounds__(128) step_simple_kernel(DevParams p, Pop<D, St> fin, Pop<D, St> gin,
                                                          Pop<D, St> fout, Pop<D, St> gout,
                                                          const float* __restrict__ phi, float* __restrict__ phiu,
                                                          const float* __restrict__ us_in, float* __restrict__ us_out)
{
    constexpr int Q = Lat<D>::Q;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int x, y, z;
    cell_xyz(p, i, x, y, z);
    float nh[Q], nl[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const long long j = nbr_index<D>(p, a, x, y, z);
        nh[a] = phi[j];
        nl[a] = phi[p.N + j];
    }
    float grad[3], lap;
    stencil_from_nb<D>(nh, nl, grad, lap);
    float fr[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) fr[a] = pulled_value<D, St>(p, fin, a, x, y, z, i);
    FlowMoments m;
    flow_moments<D>(m, fr);
    CellState s;
    float dh[27];
    if constexpr (!PR && !St::shifted) {
        if (p.flags & kFlagDivU) {  // the w cs2 rho div(u) term of Xi (Sec. 2.3)
            flow_collide<D, true>(p, nh[Q / 2], grad, lap, m, s, dh, div_stored<D>(p, us_in, x, y, z));
            for (int k = 0; k < D; ++k) us_out[k * p.N + i] = s.u[k];
            float gd[Q];
#pragma unroll
            for (int a = 0; a < Q; ++a) gd[a] = pulled_value<D, St>(p, gin, a, x, y, z, i);
            collide_outputs<D, false, true>(p, s, DhArray{dh}, m, GFromArray{gd}, nh[Q / 2], nl[Q / 2],
                                            SoAOut{fout.base + i, p.N}, SoAOut{gout.base + i, p.N});
            return;
        }
    }
    flow_collide<D>(p, nh[Q / 2], grad, lap, m, s, dh);
    constexpr int QG = PhaseLat<D, PR>::Q;
    float gr[QG];
#pragma unroll
    for (int r = 0; r < QG; ++r) {
        int slot;
        const long long c = pull_src_g<D, PR>(p, r, x, y, z, i, slot);
        gr[r] = gin.load(slot, c);
    }
    if constexpr (PR) {
        collide_outputs<D, true>(p, s, DhArray{dh}, m, GFromArray{gr}, nh[Q / 2], nl[Q / 2], SoAOut{fout.base + i, p.N},
                                 SoAOut{gout.base + i, p.N}, PhiUStep<D>{p, phiu, i});
    } else if constexpr (St::shifted) {
        float off_f, off_g;
        rest_offsets<D, St>(p, s, dh, GFromArray{gr}, off_f, off_g);
        collide_outputs<D>(p, s, DhArray{dh}, m, GFromArray{gr}, nh[Q / 2], nl[Q / 2],
                           EncSoA<D, St>{fout.base + i, (unsigned short*)(fout.base + p.N) + i, p.N, off_f, 0.f,
                                         code_seed(p, i, 0)},
                           EncSoA<D, St>{gout.base + i, (unsigned short*)(gout.base + p.N) + i, p.N, off_g, 0.f,
                                         code_seed(p, i, 1)});
    } else {
        collide_outputs<D>(p, s, DhArray{dh}, m, GFromArray{gr}, nh[Q / 2], nl[Q / 2], SoAOut{fout.base + i, p.N},
                           SoAOut{gout.base + i, p.N});
    }
}

static unsigned grid_for(long long n, int block) { return (unsigned)((n + block - 1) / block); }

// Calls F::template run<D, St, PR>() for the handle's lattice, storage form
// and phase lattice (PR: reduced, FP32 storage only).
template <class F>
static cudaError_t dispatch(const lbmp_handle* h, const F& f)
{
    const int st = h->params.storage;
    if (h->D == 3) {
        if (st == LBMP_FP16_SHIFTED) return f.template run<3, StoreF16, false>();
        if (st == LBMP_BF16_SHIFTED) return f.template run<3, StoreBF16, false>();
        return h->reduced ? f.template run<3, StoreF32, true>() : f.template run<3, StoreF32, false>();
    }
    if (st == LBMP_FP16_SHIFTED) return f.template run<2, StoreF16, false>();
    if (st == LBMP_BF16_SHIFTED) return f.template run<2, StoreBF16, false>();
    return h->reduced ? f.template run<2, StoreF32, true>() : f.template run<2, StoreF32, false>();
}

template <int D, class St>
static Pop<D, St> pop_of(const lbmp_handle* h, float* base)
{
    return Pop<D, St>{base, h->N};
}

struct PhiPassL {
    lbmp_handle* h;
    template <int D, class St, bool PR>
    cudaError_t run() const
    {
        const int B = 256;
        phi_pass_kernel<D, St, PR><<<grid_for(h->N, B), B, 0, h->stream>>>(
            h->dp, pop_of<D, St>(h, h->g[h->parity]), phi_buf(h));
        return cudaGetLastError();
    }
};

cudaError_t launch_phi_pass(lbmp_handle* h) { return dispatch(h, PhiPassL{h}); }

struct StepSimpleL {
    lbmp_handle* h;
    template <int D, class St, bool PR>
    cudaError_t run() const
    {
        const int B = 128;
        const int s = h->parity, d = 1 - h->parity;
        step_simple_kernel<D, St, PR><<<grid_for(h->N, B), B, 0, h->stream>>>(
            h->dp, pop_of<D, St>(h, h->f[s]), pop_of<D, St>(h, h->g[s]), pop_of<D, St>(h, h->f[d]),
            pop_of<D, St>(h, h->g[d]), h->phi, h->phiu, h->uvel[s], h->uvel[d]);
        return cudaGetLastError();
    }
};

cudaError_t launch_step_simple(lbmp_handle* h)
{
    // the pair writes the other population sets while it reads phi: phi must
    // have an array of its own (allocated when the pair is selected)
    if (!h->phi) return cudaErrorInvalidValue;
    cudaError_t e = launch_phi_pass(h);
    if (e != cudaSuccess) return e;
    return dispatch(h, StepSimpleL{h});
}

// rho, u and p_h of one cell as the step computes them (defined below);
// ustore: the stored previous velocity for the divergence term, or null
template <int D, class St>
__device__ void cell_macro(const DevParams& p, const Pop<D, St>& f, const float* __restrict__ phi, int x, int y,
                           int z, long long i, float& rho, float u[3], float& ph, const float* __restrict__ ustore);

// ---------------------------------------------------- initial conditions
// splitmix64 (Steele, Lea & Flood 2014): output of the (counter+1)-th call of
// the generator whose state starts at seed.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long counter)
{
    unsigned long long z = seed + (counter + 1ULL) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

struct InitArgs {
    double a[8];
    int nargs;
    double W, rho_l, rho_h, sigma, U_ref, g;
    unsigned long long seed;
    int case_id;
};

__device__ __forceinline__ double tanh_prof(double d, double W) { return 0.5 * (1.0 + tanh(2.0 * d / W)); }

// Initial conditions (reading A18): tanh phi profiles, f' = f'_eq(p, rho, u),
// g = g_eq(phi, u), written to the FP32 slots the next step pulls from, or
// (cf != null) as canonical FP64 arrays [a][cell] for the shifted encoder.
template <int D, bool PR>
__global__ void init_kernel(DevParams p, InitArgs A, float* __restrict__ f, float* __restrict__ g,
                            double* __restrict__ cf, double* __restrict__ cg)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int x, y, z;
    cell_xyz(p, i, x, y, z);
    // global position of the cell (a z-slab holds planes zoff.. of an axis of
    // nzg planes; a plain domain has zoff = 0, nzg = nz) and its global index,
    // which seeds the velocity noise
    int zg = z;
    long long gi = i;
    if (D == 3) {
        zg = z + p.zoff;
        zg = zg < 0 ? zg + p.nzg : (zg >= p.nzg ? zg - p.nzg : zg);
        gi = ((long long)zg * p.ny + y) * p.nx + x;
    }
    const int n[3] = {p.nx, p.ny, D == 3 ? p.nzg : p.nz};
    const double pos[3] = {(double)x, (double)y, (double)zg};
    const int v = D - 1;
    const double hv = pos[v];
    const double PI = 3.14159265358979323846;
    double phi = 0.0, pr = 0.0, u[3] = {0.0, 0.0, 0.0}, noise = 0.0;
    switch (A.case_id) {
    case LBMP_CASE_RT: {
        double hh = A.a[0] + A.a[1] * cos(2.0 * PI * x / n[0]);
        if (D == 3) hh += A.a[1] * cos(2.0 * PI * y / n[1]);
        phi = tanh_prof(hv - hh, A.W);
        noise = A.a[2];
        if (A.a[3] != 0.0) {
            // hydrostatic start: dp/dz = -(rho - rho_bar) g along the column, i.e.
            // p = -g (rho_h - rho_l) (W/4) ln cosh(2 (z - h)/W), zero at the interface
            const double t = fabs(2.0 * (hv - hh) / A.W);
            const double lncosh = t + log1p(exp(-2.0 * t)) - log(2.0);
            pr = -A.g * (A.rho_h - A.rho_l) * 0.25 * A.W * lncosh;
        }
        break;
    }
    case LBMP_CASE_DROP_STATIC: {
        double r2 = 0.0;
        for (int k = 0; k < D; ++k) {
            const double dx = pos[k] - (double)(n[k] / 2);
            r2 += dx * dx;
        }
        phi = tanh_prof(A.a[0] - sqrt(r2), A.W);
        if (A.a[1] != 0.0) pr = (D == 3 ? 2.0 : 1.0) * A.sigma / A.a[0] * phi;
        noise = A.a[2];
        break;
    }
    case LBMP_CASE_FLAT:
        phi = tanh_prof(fmin(pos[0] - A.a[0], A.a[1] - pos[0]), A.W);
        noise = A.a[2];
        break;
    case LBMP_CASE_POISEUILLE:
        phi = tanh_prof(0.5 * (n[v] - 1) - hv, A.W);
        noise = A.a[0];
        break;
    case LBMP_CASE_DROP_SHEET: {
        const double Dd = A.a[0], sheet = A.a[1], U0 = A.a[2];
        const double zc = sheet + 0.5 * Dd + 2.0 * A.W;
        double r2 = 0.0;
        for (int k = 0; k < D; ++k) {
            // the drop's axis: at n/2, or at the coordinate given (on a
            // symmetry face, -0.5, for a half domain)
            const double c0 = (k == v) ? zc : (A.nargs > 4 ? A.a[4] : (double)(n[k] / 2));
            const double dx = pos[k] - c0;
            r2 += dx * dx;
        }
        const double d_drop = 0.5 * Dd - sqrt(r2);
        phi = tanh_prof(fmax(d_drop, sheet - hv), A.W);
        u[v] = -U0 * tanh_prof(d_drop, A.W);
        noise = A.a[3];
        break;
    }
    case LBMP_CASE_SHEAR_WAVE:
        phi = 1.0;
        u[0] = A.a[0] * sin(2.0 * PI * y / n[1]);
        noise = A.a[1];
        break;
    default:  // LBMP_CASE_UNIFORM
        phi = A.a[0];
        pr = A.a[1];
        u[0] = A.a[2];
        u[1] = A.a[3];
        u[2] = (D == 3) ? A.a[4] : 0.0;
        break;
    }
    if (noise != 0.0) {
        for (int k = 0; k < D; ++k) {
            const double r = (double)(splitmix64(A.seed, 3ULL * (unsigned long long)gi + k) >> 11) *
                             (1.0 / 9007199254740992.0);
            u[k] += noise * A.U_ref * (2.0 * r - 1.0) * phi;
        }
    }
    const double rho = A.rho_l + (A.rho_h - A.rho_l) * phi;
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
    for (int a = 0; a < Lat<D>::Q; ++a) {
        const double w = w1d(Lat<D>::cx(a)) * w1d(Lat<D>::cy(a)) * (D == 3 ? w1d(Lat<D>::cz(a)) : 1.0);
        const double cu = Lat<D>::cx(a) * u[0] + Lat<D>::cy(a) * u[1] + Lat<D>::cz(a) * u[2];
        // Gamma - w = w [c.u/cs2 + ((c.u)^2 - cs2 u^2)/(2 cs4)]
        const double gdev = w * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
        const double fe = w * pr + rho * (1.0 / 3.0) * gdev;  // f'_eq (Sec. 2.3)
        const double ge = phi * (w + gdev);                    // g_eq (Sec. 2.2)
        if (cf) {
            cf[(long long)a * p.N + i] = fe;
            cg[(long long)a * p.N + i] = ge;
        } else if (has_pull_slot<D>(p, a, z)) {
            const long long slot = pull_index<D>(p, a, x, y, z, i);
            f[slot] = (float)fe;
            if (!PR) g[slot] = (float)ge;
        }
    }
    if constexpr (PR) {
        // reduced phase lattice: first-order equilibrium w phi (1 + c.u/cs2) (Sec. 2.2)
        constexpr int C = PhaseLat<D, true>::C;
#pragma unroll
        for (int r = 0; r < PhaseLat<D, true>::Q; ++r) {
            const int a = PhaseLat<D, true>::full(r);
            const double w = (r == C) ? (D == 3 ? 0.25 : 1.0 / 3.0) : (D == 3 ? 0.125 : 1.0 / 6.0);
            const double cu = Lat<D>::cx(a) * u[0] + Lat<D>::cy(a) * u[1] + Lat<D>::cz(a) * u[2];
            if (!has_pull_slot<D>(p, a, z)) continue;
            int slot;
            const long long c = pull_src_g<D, true>(p, r, x, y, z, i, slot);
            g[(long long)slot * p.N + c] = (float)(w * phi * (1.0 + cu * (D == 3 ? 4.0 : 3.0)));
        }
    }
}

// Reduced phase lattice: phi u of every cell from the current state (the u
// the next step's closure computes), the previous value before the first step
// after init / set_state.  Needs the phi pass first.
// The same for the stored velocity of the divergence term (kFlagDivU): the
// previous velocity before the first step is the current one.
template <int D>
__global__ void phiu_reset_kernel(DevParams p, Pop<D, StoreF32> f, const float* __restrict__ phi,
                                  float* __restrict__ phiu, float* __restrict__ ustore)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int x, y, z;
    cell_xyz(p, i, x, y, z);
    float rho, u[3], ph;
    cell_macro<D, StoreF32>(p, f, phi, x, y, z, i, rho, u, ph, nullptr);
    for (int k = 0; k < D; ++k) {
        if (phiu) phiu[k * p.N + i] = phi[i] * u[k];
        if (ustore) ustore[k * p.N + i] = u[k];
    }
}

cudaError_t launch_init(lbmp_handle* h, int case_id, const double* args, int nargs, unsigned long long seed)
{
    InitArgs A;
    for (int k = 0; k < 8; ++k) A.a[k] = args[k];
    A.nargs = nargs;
    A.W = h->der.W;
    A.rho_l = h->der.rho_l;
    A.rho_h = h->der.rho_h;
    A.sigma = h->der.sigma;
    A.U_ref = h->der.U_ref;
    A.g = h->der.g_accel;
    A.seed = seed;
    A.case_id = case_id;
    const int B = 128;
    if (h->params.storage == LBMP_FP32) {
        float *f = h->f[h->parity], *g = h->g[h->parity];
        const unsigned grid = grid_for(h->N, B);
        if (h->D == 3 && h->reduced)
            init_kernel<3, true><<<grid, B, 0, h->stream>>>(h->dp, A, f, g, nullptr, nullptr);
        else if (h->D == 3)
            init_kernel<3, false><<<grid, B, 0, h->stream>>>(h->dp, A, f, g, nullptr, nullptr);
        else if (h->reduced)
            init_kernel<2, true><<<grid, B, 0, h->stream>>>(h->dp, A, f, g, nullptr, nullptr);
        else
            init_kernel<2, false><<<grid, B, 0, h->stream>>>(h->dp, A, f, g, nullptr, nullptr);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = launch_phiu_reset(h);
        return e;
    }
    // shifted storage: canonical FP64 state first, then the per-cell encoder
    const size_t n = (size_t)h->Q * (size_t)h->N;
    double* c = nullptr;
    cudaError_t e = cudaMallocAsync(&c, 2 * n * sizeof(double), h->stream);
    if (e != cudaSuccess) return e;
    if (h->D == 3)
        init_kernel<3, false><<<grid_for(h->N, B), B, 0, h->stream>>>(h->dp, A, nullptr, nullptr, c, c + n);
    else
        init_kernel<2, false><<<grid_for(h->N, B), B, 0, h->stream>>>(h->dp, A, nullptr, nullptr, c, c + n);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_set_state(h, c, c + n);
    cudaFreeAsync(c, h->stream);
    return e;
}

// ------------------------------------------------------ state exchange
// canonical (post-streaming, [a][cell]) FP64 <- stored state
template <int D, class St, bool PR>
__global__ void get_state_kernel(DevParams p, Pop<D, St> f, Pop<D, St> g, double* cf, double* cg)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int x, y, z;
    cell_xyz(p, i, x, y, z);
#pragma unroll
    for (int a = 0; a < Lat<D>::Q; ++a)
        if (cf) cf[(long long)a * p.N + i] = (double)pulled_value<D, St>(p, f, a, x, y, z, i);
#pragma unroll
    for (int r = 0; r < PhaseLat<D, PR>::Q; ++r) {
        int slot;
        const long long c = pull_src_g<D, PR>(p, r, x, y, z, i, slot);
        if (cg) cg[(long long)r * p.N + i] = (double)g.load(slot, c);
    }
}

// stored FP32 state <- canonical FP64 (one thread per reading cell)
template <int D, bool PR>
__global__ void set_state_f32_kernel(DevParams p, float* f, float* g, const double* cf, const double* cg)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= p.N) return;
    int x, y, z;
    cell_xyz(p, i, x, y, z);
#pragma unroll
    for (int a = 0; a < Lat<D>::Q; ++a)
        if (has_pull_slot<D>(p, a, z)) f[pull_index<D>(p, a, x, y, z, i)] = (float)cf[(long long)a * p.N + i];
#pragma unroll
    for (int r = 0; r < PhaseLat<D, PR>::Q; ++r) {
        if (!has_pull_slot<D>(p, PhaseLat<D, PR>::full(r), z)) continue;
        int slot;
        const long long c = pull_src_g<D, PR>(p, r, x, y, z, i, slot);
        g[(long long)slot * p.N + c] = (float)cg[(long long)r * p.N + i];
    }
}

// Shifted encoding of one writer cell from the canonical values v[a] of the
// slots it owns (FP64 arithmetic; R from the exact total, see Pop).  Codes
// round to nearest here: this rounds a set state once, where the step's
// stochastic rounding guards against a bias repeated every step.
template <int D, class St>
__device__ void encode_cell(const Pop<D, St>& set, long long j, const double* v)
{
    constexpr int Q = Lat<D>::Q, C = Q / 2;
    double T = 0.0;
    for (int a = 0; a < Q; ++a) T += v[a];
    const double rC = v[C] / (double)wint<D>(C);
    unsigned short* q = (unsigned short*)(set.base + set.N);
    double sum = 0.0;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        if (a == C) continue;
        const double W = (double)wint<D>(a);
        const unsigned short c = St::enc((float)((v[a] / W - rC) * (double)St::S));
        q[(a - (a > C)) * set.N + j] = c;
        sum += W * (double)St::s * (double)St::dec(c);
    }
    set.base[j] = (float)((T - sum) / (double)wden<D>());
}

template <int D, class St>
__global__ void set_state_shifted_kernel(DevParams p, Pop<D, St> f, Pop<D, St> g, const double* cf,
                                         const double* cg)
{
    constexpr int Q = Lat<D>::Q;
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= p.N) return;
    int x, y, z;
    cell_xyz(p, j, x, y, z);
    double vf[Q], vg[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        int dir;
        const long long r = push_dst<D>(p, a, x, y, z, j, dir);
        vf[a] = cf[(long long)dir * p.N + r];
        vg[a] = cg[(long long)dir * p.N + r];
    }
    encode_cell<D, St>(f, j, vf);
    encode_cell<D, St>(g, j, vg);
}

struct SetStateL {
    lbmp_handle* h;
    const double *cf, *cg;
    template <int D, class St, bool PR>
    cudaError_t run() const
    {
        const int B = 128;
        float *f = h->f[h->parity], *g = h->g[h->parity];
        if constexpr (St::shifted)
            set_state_shifted_kernel<D, St><<<grid_for(h->N, B), B, 0, h->stream>>>(
                h->dp, pop_of<D, St>(h, f), pop_of<D, St>(h, g), cf, cg);
        else
            set_state_f32_kernel<D, PR><<<grid_for(h->N, B), B, 0, h->stream>>>(h->dp, f, g, cf, cg);
        return cudaGetLastError();
    }
};

struct GetStateL {
    lbmp_handle* h;
    double *cf, *cg;
    template <int D, class St, bool PR>
    cudaError_t run() const
    {
        const int B = 128;
        get_state_kernel<D, St, PR><<<grid_for(h->N, B), B, 0, h->stream>>>(
            h->dp, pop_of<D, St>(h, h->f[h->parity]), pop_of<D, St>(h, h->g[h->parity]), cf, cg);
        return cudaGetLastError();
    }
};

cudaError_t launch_set_state(lbmp_handle* h, const double* dev_f, const double* dev_g)
{
    cudaError_t e = dispatch(h, SetStateL{h, dev_f, dev_g});
    if (e == cudaSuccess) e = launch_phiu_reset(h);
    return e;
}

cudaError_t launch_phiu_reset(lbmp_handle* h)
{
    if (!h->reduced && !h->divu) return cudaSuccess;
    cudaError_t e = launch_phi_pass(h);
    if (e != cudaSuccess) return e;
    const int B = 128;
    if (h->D == 3)
        phiu_reset_kernel<3><<<grid_for(h->N, B), B, 0, h->stream>>>(h->dp, pop_of<3, StoreF32>(h, h->f[h->parity]),
                                                                     phi_buf(h), h->phiu, h->uvel[h->parity]);
    else
        phiu_reset_kernel<2><<<grid_for(h->N, B), B, 0, h->stream>>>(h->dp, pop_of<2, StoreF32>(h, h->f[h->parity]),
                                                                     phi_buf(h), h->phiu, h->uvel[h->parity]);
    return cudaGetLastError();
}

cudaError_t launch_get_state(lbmp_handle* h, double* dev_f, double* dev_g)
{
    return dispatch(h, GetStateL{h, dev_f, dev_g});
}

// ---------------------------------------------------------- observables
// rho, u and p_h = P + cs2 u.grad(rho)/2 of one cell, as in the step.
template <int D, class St>
__device__ void cell_macro(const DevParams& p, const Pop<D, St>& f, const float* __restrict__ phi, int x, int y,
                           int z, long long i, float& rho, float u[3], float& ph, const float* __restrict__ ustore)
{
    constexpr int Q = Lat<D>::Q;
    float nh[Q], nl[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const long long j = nbr_index<D>(p, a, x, y, z);
        nh[a] = phi[j];
        nl[a] = phi[p.N + j];
    }
    float grad[3], lap;
    stencil_from_nb<D>(nh, nl, grad, lap);
    float fr[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) fr[a] = pulled_value<D, St>(p, f, a, x, y, z, i);
    FlowMoments m;
    flow_moments<D>(m, fr);
    CellState s;
    float inv_rho, nu;
    if (ustore)
        rho = flow_closure<D, true>(p, nh[Q / 2], grad, lap, m, s, inv_rho, nu, div_stored<D>(p, ustore, x, y, z));
    else
        rho = flow_closure<D>(p, nh[Q / 2], grad, lap, m, s, inv_rho, nu);
    for (int k = 0; k < 3; ++k) u[k] = s.u[k];
    ph = s.ph;
}

// per-block partial sums: mass, kinetic energy, max|u|, non-finite count
template <int D, class St>
__global__ void __launch_bounds__(256) obs_partial_kernel(DevParams p, Pop<D, St> f, const float* __restrict__ phi,
                                                          double* __restrict__ part, const float* __restrict__ ustore)
{
    __shared__ double sm[4][256];
    double mass = 0.0, ke = 0.0, um = 0.0, bad = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < p.N;
         i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_xyz(p, i, x, y, z);
        if (D == 3 && (z < p.zb || z >= p.ze)) continue;  // a z-slab's ghost planes belong to its neighbours
        float rho, u[3], ph;
        cell_macro<D, St>(p, f, phi, x, y, z, i, rho, u, ph, ustore);
        const double uu = (double)u[0] * u[0] + (double)u[1] * u[1] + (double)u[2] * u[2];
        const double ph_i = (double)phi[i] + (double)phi[p.N + i];
        mass += ph_i;
        ke += 0.5 * rho * uu;
        const double un = sqrt(uu);
        if (!(un <= um)) um = un;
        if (!isfinite(ph_i) || !isfinite(uu) || !isfinite(ph)) bad += 1.0;
    }
    const int t = threadIdx.x;
    sm[0][t] = mass;
    sm[1][t] = ke;
    sm[2][t] = um;
    sm[3][t] = bad;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (t < s) {
            sm[0][t] += sm[0][t + s];
            sm[1][t] += sm[1][t + s];
            const double o = sm[2][t + s];
            if (!(o <= sm[2][t])) sm[2][t] = o;
            sm[3][t] += sm[3][t + s];
        }
        __syncthreads();
    }
    if (t == 0)
        for (int k = 0; k < 4; ++k) part[4 * blockIdx.x + k] = sm[k][0];
}

// fixed-order final reduction of the partials (deterministic for a fixed grid)
__global__ void __launch_bounds__(256) obs_final_kernel(const double* __restrict__ part, int nblocks,
                                                        double* __restrict__ out)
{
    __shared__ double sm[4][256];
    const int t = threadIdx.x;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = t; b < nblocks; b += 256) {
        acc[0] += part[4 * b];
        acc[1] += part[4 * b + 1];
        const double o = part[4 * b + 2];
        if (!(o <= acc[2])) acc[2] = o;
        acc[3] += part[4 * b + 3];
    }
    for (int k = 0; k < 4; ++k) sm[k][t] = acc[k];
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (t < s) {
            sm[0][t] += sm[0][t + s];
            sm[1][t] += sm[1][t + s];
            const double o = sm[2][t + s];
            if (!(o <= sm[2][t])) sm[2][t] = o;
            sm[3][t] += sm[3][t + s];
        }
        __syncthreads();
    }
    if (t == 0)
        for (int k = 0; k < 4; ++k) out[k] = sm[k][0];
}

// mean p_h over the 3^D block at a probe cell (one block of threads per probe)
template <int D, class St>
__global__ void probe_kernel(DevParams p, Pop<D, St> f, const float* __restrict__ phi, int px, int py, int pz, int qx,
                             int qy, int qz, double* __restrict__ out, const float* __restrict__ ustore)
{
    __shared__ double sm[32];
    const int t = threadIdx.x;
    const int npts = (D == 3) ? 27 : 9;
    const int cx = blockIdx.x == 0 ? px : qx, cy = blockIdx.x == 0 ? py : qy, cz = blockIdx.x == 0 ? pz : qz;
    double v = 0.0;
    if (t < npts) {
        const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = (D == 3) ? t / 9 - 1 : 0;
        const int x = wrap_h(cx + dx, p.nx);
        int y, z;
        if (D == 3) {
            y = wrap_h(cy + dy, p.ny);
            z = wrap_v(cz + dz, p.nz, p.vert_periodic);
        } else {
            y = wrap_v(cy + dy, p.ny, p.vert_periodic);
            z = 0;
        }
        const long long i = ((long long)z * p.ny + y) * p.nx + x;
        float rho, u[3], ph;
        cell_macro<D, St>(p, f, phi, x, y, z, i, rho, u, ph, ustore);
        v = ph;
    }
    sm[t] = v;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int k = 0; k < npts; ++k) s += sm[k];
        out[blockIdx.x] = s / npts;
    }
}

// phi on the spike column (nx/2, ny/2) and the bubble column (0, 0)
template <int D>
__global__ void column_kernel(DevParams p, const float* __restrict__ phi, double* __restrict__ out)
{
    const int nv = (D == 3) ? p.nz : p.ny;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nv) return;
    long long is, ib;
    if (D == 3) {
        is = ((long long)k * p.ny + p.ny / 2) * p.nx + p.nx / 2;
        ib = (long long)k * p.ny * p.nx;
    } else {
        is = (long long)k * p.nx + p.nx / 2;
        ib = (long long)k * p.nx;
    }
    out[k] = (double)phi[is] + (double)phi[p.N + is];
    out[nv + k] = (double)phi[ib] + (double)phi[p.N + ib];
}

struct ObsL {
    lbmp_handle* h;
    double* out;
    bool full;  // false: mass and the other reductions only
    template <int D, class St, bool>
    cudaError_t run() const
    {
        const Pop<D, St> f = pop_of<D, St>(h, h->f[h->parity]);
        const float* us = h->uvel[h->parity];  // the velocity the next step's div(u) uses, or null
        const float* phi = phi_buf(h);
        obs_partial_kernel<D, St><<<h->red_blocks, 256, 0, h->stream>>>(h->dp, f, phi, h->red, us);
        obs_final_kernel<<<1, 256, 0, h->stream>>>(h->red, h->red_blocks, out);
        if (full) {
            const int nv = (D == 3) ? h->grid.nz : h->grid.ny;
            const int* pr = h->probe;
            probe_kernel<D, St><<<2, 32, 0, h->stream>>>(h->dp, f, phi, pr[0], pr[1], D == 3 ? pr[2] : 0, 0, 0,
                                                         0, out + 4, us);
            column_kernel<D><<<grid_for(nv, 128), 128, 0, h->stream>>>(h->dp, phi, out + 16);
        }
        return cudaGetLastError();
    }
};

cudaError_t launch_observables(lbmp_handle* h, double* dev_out)
{
    cudaError_t e = launch_phi_pass(h);
    if (e != cudaSuccess) return e;
    return dispatch(h, ObsL{h, dev_out, true});
}

cudaError_t launch_mass(lbmp_handle* h, double* dev_out4)
{
    cudaError_t e = launch_phi_pass(h);
    if (e != cudaSuccess) return e;
    return dispatch(h, ObsL{h, dev_out4, false});
}

}  // namespace lbmp
