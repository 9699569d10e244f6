// lbmp_common.cuh -- lattice traits, device parameters and the per-cell
// arithmetic of the coupled update (Hosseini, Safari & Thevenin, arXiv
// 2101.06769, Sec. 2.2 and 2.3), shared by every step kernel of the library.
//
// All arithmetic is FP32.  The flow collision is written in "deviation
// form": every quantity that enters a stored population is formed as a small
// deviation from the rest state, so that FP32 keeps full relative precision
// on f' (whose values are O(p_h) and O(rho cs2 u), far below the O(1) rest
// weights).  The form is algebraically identical to the general cumulant
// path of Sec. 2.3 because every rate other than the shear rate is one:
//   * the post-collision cumulants of order >= 3 vanish, so the post-collision
//     central moments are the Gaussian (Isserlis) moments of the relaxed
//     second-order tensor kappa* = cs2 I + delta*;
//   * the product-form equilibrium E(u) has the Gaussian moments of cs2 I, so
//     h* - E(u) is the per-axis (Kronecker) inverse of the 13 non-zero moment
//     differences, and E(u) - w is a telescoped product of per-axis terms.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

// 1: the pair loops of phase_outputs / flow_outputs keep their memory
// operations in program order (a compiler barrier per pair), so that the
// compiler does not hoist the loads of later pairs; this lowers the register
// footprint of a kernel built for four CTAs per SM at no change in results
#ifndef LBMP_OUT_ORDERED
#define LBMP_OUT_ORDERED 0
#endif

namespace lbmp {

__device__ __forceinline__ void out_pair_done()
{
#if LBMP_OUT_ORDERED
    asm volatile("" ::: "memory");
#endif
}

__host__ __device__ constexpr double w1d(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }

// Velocity set {-1,0,1}^D in the exchange order a = (cx+1) + 3(cy+1) + 9(cz+1)
// with the tensorised D1Q3 Gauss-Hermite weights (cs2 = 1/3, Sec. 2.2).
template <int D>
struct Lat;

template <>
struct Lat<3> {
    static constexpr int Q = 27;
    __host__ __device__ static constexpr int cx(int a) { return a % 3 - 1; }
    __host__ __device__ static constexpr int cy(int a) { return (a / 3) % 3 - 1; }
    __host__ __device__ static constexpr int cz(int a) { return a / 9 - 1; }
    __host__ __device__ static constexpr float w(int a) { return (float)(w1d(cx(a)) * w1d(cy(a)) * w1d(cz(a))); }
    __host__ __device__ static constexpr int opp(int a) { return 26 - a; }
    __host__ __device__ static constexpr int mx(int a) { return a - 2 * cx(a); }  // x velocity reversed
};

template <>
struct Lat<2> {
    static constexpr int Q = 9;
    __host__ __device__ static constexpr int cx(int a) { return a % 3 - 1; }
    __host__ __device__ static constexpr int cy(int a) { return a / 3 - 1; }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr float w(int a) { return (float)(w1d(cx(a)) * w1d(cy(a))); }
    __host__ __device__ static constexpr int opp(int a) { return 8 - a; }
    __host__ __device__ static constexpr int mx(int a) { return a - 2 * cx(a); }  // x velocity reversed
};

constexpr float kCs2 = 1.0f / 3.0f;

enum : unsigned {
    kFlagWeLight = 1u << 0,
    kFlagDynamicVisc = 1u << 1,
    kFlagUniformForce = 1u << 2,
    kFlagPhaseReduced = 1u << 3,
    kFlagDivU = 1u << 4,
};

// Lattice of the phase field g.  PR = false: the flow lattice with the
// second-order equilibrium.  PR = true: the rest and face directions only
// (D3Q7: weights 1/4, 1/8, cs2 = 1/4; D2Q5: 1/3, 1/6, cs2 = 1/3), with the
// first-order equilibrium w phi (1 + c.u/cs2) and the correction term
// C_bar = lambda (w/cs2) c . d/dt(phi u) that Sec. 2.2 gives for it.  Slot r
// holds the flow-lattice direction full(r); the slots keep the canonical
// order, so opposite(r) = Q-1-r.
template <int D, bool PR>
struct PhaseLat {
    static constexpr int Q = PR ? 2 * D + 1 : Lat<D>::Q;
    static constexpr int C = Q / 2;
    __host__ __device__ static constexpr int full(int r)
    {
        if (!PR) return r;
        if (D == 3) return r == 3 ? 13 : (r < 3 ? (r == 0 ? 4 : (r == 1 ? 10 : 12)) : (r == 4 ? 14 : (r == 5 ? 16 : 22)));
        return r == 2 ? 4 : (r < 2 ? (r == 0 ? 1 : 3) : (r == 3 ? 5 : 7));
    }
    __host__ __device__ static constexpr float w(int r)
    {
        if (!PR) return Lat<D>::w(r);
        return r == C ? (D == 3 ? 0.25f : 1.f / 3.f) : (D == 3 ? 0.125f : 1.f / 6.f);
    }
    static constexpr float inv_cs2 = (PR && D == 3) ? 4.f : 3.f;
};

// Everything a step kernel needs, by value (fits the kernel-parameter space).
struct DevParams {
    int nx, ny, nz;         // nz = 1 in 2-D
    int vert_periodic;      // vertical axis periodic (1) or walled (0)
    // Vertical axis of a z-slab (one rank's planes of a domain decomposed
    // along z; equal to the plain values otherwise): half-way bounce-back
    // wall below plane 0 / above plane nz-1 (wall_lo / wall_hi), the planes
    // [zb, ze) the step updates (the others are ghost planes filled by the
    // exchange), the global index of plane 0 (zoff) and the global extent
    // (nzg).  A slab's local axis is periodic in the index arithmetic, but no
    // updated plane or staged ghost ever pulls across its ends.
    int wall_lo, wall_hi;
    int zb, ze;
    int zoff, nzg;
    // In-place AA storage (LBMP_FLAG_AA: one population set each for f' and
    // g): 0 = two sets (the stored value of direction a at cell i is the
    // post-collision value of the upstream cell); 1 = AA, natural phase (the
    // streamed value of a at i is A[a][i]); 2 = AA, swapped phase (it is
    // A[opp(a)][i - c_a], or A[a][i] across a wall)
    int aa;
    // D2Q9 only: the x axis is a symmetry axis (reading A28: half-way
    // specular reflection at both faces, the phi ghost equal to the boundary
    // cell) instead of periodic
    int sym_x;
    long long N;            // cells
    float rho_l, drho, rho_bar;
    float nu_h, nu_l, eta_h, eta_l;
    float beta2, kappa;     // 2 beta, kappa of the chemical potential
    float inv_tau_phi;      // 1/tau_bar_phi
    float lam_sharp;        // lambda_phi * 4 / W
    float lam_corr;         // lambda_phi / cs2 of the phase lattice (reduced phase lattice)
    float g_accel, force_x;
    unsigned flags;
    int* status;            // device status word of the handle (kStatus* bits), or null
    unsigned long long wait_ns;  // bound of every wait of a step kernel (nanoseconds)
    unsigned step;               // index of the step being taken (seeds the stochastic rounding of BF16 codes)
    unsigned test_extra_tx;      // test only: extra bytes expected per staged plane (its wait runs out)
};

// bits of the device status word
constexpr int kStatusWaitTimeout = 1;  // a bounded wait of a step kernel ran out

// Paired FP32 arithmetic (sm_100+ FFMA2/FADD2/FMUL2): one instruction
// updates both lanes, each lane rounded exactly as its scalar counterpart.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
// TwoSum (Knuth) on both lanes: hi + lo accumulates v exactly
__device__ __forceinline__ void two_sum2(float2& hi, float2& lo, float2 v)
{
    const float2 t = add2(hi, v);
    const float2 bb = add2(t, neg2(hi));
    lo = add2(lo, add2(add2(hi, neg2(add2(t, neg2(bb)))), add2(v, neg2(bb))));
    hi = t;
}

// directions a < Q/2 in order of decreasing weight (faces, edges, corners)
template <int D>
__host__ __device__ constexpr int by_weight(int k)  // k-th direction a < Q/2 by decreasing weight
{
    constexpr int o3[13] = {4, 10, 12, 1, 3, 5, 7, 9, 11, 0, 2, 6, 8};
    constexpr int o2[4] = {1, 3, 0, 2};
    return D == 3 ? o3[k] : o2[k];
}

// ----------------------------------------------------------- pull helpers
// Post-streaming population a at cell (x,y,z) lives in the buffer written by
// the previous step at the upstream cell x - c_a (pull); across a half-way
// bounce-back wall it is the opposite population of the cell itself.
// Returns the cell holding it and sets dir to the direction slot.
template <int D>
__device__ __forceinline__ long long pull_src(const DevParams& p, int a, int x, int y, int z, long long self,
                                              int& dir)
{
    const int cx = Lat<D>::cx(a), cy = Lat<D>::cy(a), cz = Lat<D>::cz(a);
    int xs = x - cx;
    xs = xs < 0 ? xs + p.nx : (xs >= p.nx ? xs - p.nx : xs);
    dir = a;
    if (D == 3) {
        if (p.aa == 1) return self;  // AA, natural phase: own cell, own direction
        int ys = y - cy;
        ys = ys < 0 ? ys + p.ny : (ys >= p.ny ? ys - p.ny : ys);
        int zs = z - cz;
        if (zs < 0 || zs >= p.nz) {
            if (zs < 0 ? p.wall_lo : p.wall_hi) {
                // across a wall: the cell's own opposite value (two sets), or
                // its own value of a (AA swapped phase)
                dir = p.aa ? a : Lat<D>::opp(a);
                return self;
            }
            zs = zs < 0 ? zs + p.nz : zs - p.nz;
        }
        if (p.aa) dir = Lat<D>::opp(a);  // AA swapped phase: the upstream cell's opposite slot
        return ((long long)zs * p.ny + ys) * p.nx + xs;
    } else {
        int ys = y - cy;
        if (ys < 0 || ys >= p.ny) {
            if (!p.vert_periodic) {
                dir = Lat<D>::opp(a);
                return self;
            }
            ys = ys < 0 ? ys + p.ny : ys - p.ny;
        }
        if (p.sym_x && (x - cx < 0 || x - cx >= p.nx)) {
            // across a symmetry face: the cell's own column, the value that
            // left it with the mirrored x velocity
            dir = Lat<D>::mx(a);
            return (long long)ys * p.nx + x;
        }
        return (long long)ys * p.nx + xs;
    }
}

// A z-slab's ghost cell whose pull source lies across a local end without a
// wall has no slot in this slab (the neighbour's planes hold it): writers of
// the state skip it instead of wrapping onto the opposite end, where the
// wrapped index belongs to another cell (a wall plane's bounce-back slot,
// for one).  Always true for a plain domain (zb = 0, ze = nz).
template <int D>
__device__ __forceinline__ bool has_pull_slot(const DevParams& p, int a, int z)
{
    if (D != 3) return true;
    const int zs = z - Lat<D>::cz(a);
    if (zs < 0) return p.wall_lo || p.zb == 0;
    if (zs >= p.nz) return p.wall_hi || p.ze == p.nz;
    return true;
}

template <int D>
__device__ __forceinline__ long long pull_index(const DevParams& p, int a, int x, int y, int z, long long self)
{
    int dir;
    const long long c = pull_src<D>(p, a, x, y, z, self, dir);
    return (long long)dir * p.N + c;
}

// pull_src / push_dst for slot r of the phase lattice (slot of the opposite
// direction across a wall)
template <int D, bool PR>
__device__ __forceinline__ long long pull_src_g(const DevParams& p, int r, int x, int y, int z, long long self,
                                                int& slot)
{
    if constexpr (!PR) {
        return pull_src<D>(p, r, x, y, z, self, slot);
    } else {
        const int a = PhaseLat<D, true>::full(r);
        int dir;
        const long long c = pull_src<D>(p, a, x, y, z, self, dir);
        slot = dir == a ? r : PhaseLat<D, true>::Q - 1 - r;
        return c;
    }
}

// Inverse of pull_src: the slot (cell, a) written by the cell (x,y,z) is read
// as population dir of the returned cell (downstream x + c_a, or the cell
// itself in the opposite direction when x + c_a lies across a wall).
template <int D>
__device__ __forceinline__ long long push_dst(const DevParams& p, int a, int x, int y, int z, long long self,
                                              int& dir)
{
    const int cx = Lat<D>::cx(a), cy = Lat<D>::cy(a), cz = Lat<D>::cz(a);
    int xd = x + cx;
    xd = xd < 0 ? xd + p.nx : (xd >= p.nx ? xd - p.nx : xd);
    dir = a;
    if (D == 3) {
        int yd = y + cy;
        yd = yd < 0 ? yd + p.ny : (yd >= p.ny ? yd - p.ny : yd);
        int zd = z + cz;
        if (zd < 0 || zd >= p.nz) {
            if (zd < 0 ? p.wall_lo : p.wall_hi) {
                dir = Lat<D>::opp(a);
                return self;
            }
            zd = zd < 0 ? zd + p.nz : zd - p.nz;
        }
        return ((long long)zd * p.ny + yd) * p.nx + xd;
    } else {
        int yd = y + cy;
        if (yd < 0 || yd >= p.ny) {
            if (!p.vert_periodic) {
                dir = Lat<D>::opp(a);
                return self;
            }
            yd = yd < 0 ? yd + p.ny : yd - p.ny;
        }
        if (p.sym_x && (x + cx < 0 || x + cx >= p.nx)) {
            dir = Lat<D>::mx(a);
            return (long long)yd * p.nx + x;
        }
        return (long long)yd * p.nx + xd;
    }
}

template <int D, bool PR>
__device__ __forceinline__ long long push_dst_g(const DevParams& p, int r, int x, int y, int z, long long self,
                                                int& slot)
{
    if constexpr (!PR) {
        return push_dst<D>(p, r, x, y, z, self, slot);
    } else {
        const int a = PhaseLat<D, true>::full(r);
        int dir;
        const long long c = push_dst<D>(p, a, x, y, z, self, dir);
        slot = dir == a ? r : PhaseLat<D, true>::Q - 1 - r;
        return c;
    }
}

// ------------------------------------------------------------- storage
// Population storage forms (lbmp_storage).
//
// FP32: population a of cell i at base[a N + i].
//
// Shifted 16-bit (FP16 or BF16).  Every lattice weight is w_a = W_a / den
// with W_a a power of two (D3Q27: 64, 16, 4, 1 over 216; D2Q9: 16, 4, 1 over
// 36).  A cell stores one FP32 reference R at base[i] and, for each moving
// direction a, a 16-bit code q_a at ((u16*)(base + N))[slot(a) N + i] with
// slot(a) = a - (a > C).  The values are
//     moving a:  v_a = W_a (R + s q_a),        rest:  v_C = W_C R,
// so q holds only the deviation of v_a/W_a from the rest ratio v_C/W_C (the
// O(c.u) equilibrium part and the non-equilibrium part), while the O(p_h)
// pressure level of f' and the O(phi) level of g stay in the FP32 reference.
// W_a R and W_a s q_a are exact, so a decoded value is rounded once.  The
// writer encodes q_a = S (v_a/W_a - v_C/W_C) (s = 1/S a power of two that
// keeps FP16 codes of a light phase out of the subnormal range) and then sets
// R = (T - s sum_a W_a q_a)/den from the cell's total T, so the decoded
// populations of a cell add up to T to within one rounding: the 16-bit codes
// cannot bias mass or pressure.
template <int D>
__host__ __device__ constexpr float wint(int a)  // W_a = den w_a
{
    return (Lat<D>::cx(a) == 0 ? 4.f : 1.f) * (Lat<D>::cy(a) == 0 ? 4.f : 1.f) *
           ((D == 3 && Lat<D>::cz(a) == 0) ? 4.f : 1.f);
}
template <int D>
__host__ __device__ constexpr float wden()
{
    return D == 3 ? 216.f : 36.f;
}

struct StoreF32 {
    static constexpr bool stochastic = false;
    static constexpr bool shifted = false;
};
struct StoreF16 {
    static constexpr bool shifted = true;
    static constexpr bool stochastic = true;  // the step's codes are rounded stochastically (enc_sr)
    static constexpr float S = 1048576.f, s = 1.f / 1048576.f;  // 2^20
    // byte-permute selectors moving the low / high half of a word to bits 0..15
    static constexpr unsigned kSelLo = 0x4410u, kSelHi = 0x4432u;
    __device__ __forceinline__ static unsigned short enc(float q) { return __half_as_ushort(__float2half_rn(q)); }
    __device__ __forceinline__ static float dec(unsigned short c) { return __half2float(__ushort_as_half(c)); }
    // stochastic rounding: r (13 random bits) is added below the 10 bits an
    // FP16 significand keeps of q's, then q is rounded toward zero, so q
    // rounds away from zero with probability equal to the dropped fraction
    // of an ulp (exact for normal FP16 codes; the scale S keeps codes of
    // practical deviations out of the subnormal range)
    __device__ __forceinline__ static unsigned short enc_sr(float q, unsigned r)
    {
        return __half_as_ushort(__float2half_rz(__uint_as_float(__float_as_uint(q) + (r & 0x1fffu))));
    }
    __device__ __forceinline__ static float dec_word(unsigned w, unsigned sel)
    {
        return dec((unsigned short)__byte_perm(w, 0u, sel));
    }
};
struct StoreBF16 {
    static constexpr bool shifted = true;
    static constexpr bool stochastic = true;  // the step's codes are rounded stochastically (enc_sr)
    static constexpr float S = 1.f, s = 1.f;  // BF16 has the FP32 exponent range
    // selectors moving the low / high half of a word to bits 16..31 (zeros below)
    static constexpr unsigned kSelLo = 0x1044u, kSelHi = 0x3244u;
    __device__ __forceinline__ static unsigned short enc(float q)
    {
        return __bfloat16_as_ushort(__float2bfloat16_rn(q));
    }
    __device__ __forceinline__ static float dec(unsigned short c) { return __uint_as_float((unsigned)c << 16); }
    // stochastic rounding: q rounds away from zero with probability equal to
    // the dropped fraction of an ulp (r uniform in [0, 2^16)), so the stored
    // code is unbiased and an increment below half an ulp is not lost
    __device__ __forceinline__ static unsigned short enc_sr(float q, unsigned r)
    {
        return (unsigned short)((__float_as_uint(q) + (r & 0xffffu)) >> 16);
    }
    __device__ __forceinline__ static float dec_word(unsigned w, unsigned sel)
    {
        return __uint_as_float(__byte_perm(w, 0u, sel));
    }
};

// decoded value of moving population a from its code and the writer's reference
template <int D, class St>
__device__ __forceinline__ float dec_value(int a, float code_value, float R)
{
    const float W = wint<D>(a);
    return fmaf(code_value, W * St::s, W * R);
}

// One population set in device memory (layout above).
template <int D, class St>
struct Pop {
    float* base;
    long long N;
    __device__ __forceinline__ float load(int a, long long i) const
    {
        if constexpr (!St::shifted) {
            return base[a * N + i];
        } else {
            constexpr int C = Lat<D>::Q / 2;
            const float R = base[i];
            if (a == C) return wint<D>(C) * R;
            const unsigned short* q = (const unsigned short*)(base + N);
            return dec_value<D, St>(a, St::dec(q[(a - (a > C)) * N + i]), R);
        }
    }
    // the two exact parts W_a R and W_a s q_a of a shifted value (wq = 0 for the rest)
    __device__ __forceinline__ void load_parts(int a, long long i, float& wr, float& wq) const
    {
        constexpr int C = Lat<D>::Q / 2;
        const float W = wint<D>(a);
        wr = W * base[i];
        wq = 0.f;
        if (a != C) {
            const unsigned short* q = (const unsigned short*)(base + N);
            wq = St::dec(q[(a - (a > C)) * N + i]) * (W * St::s);
        }
    }
};

// phi = sum_a v_a for shifted storage, from the exact parts of each value
// (v_a = W_a R + W_a s q_a): the reference parts, of comparable size, in the
// Fast2Sum chain of phi_sum (rest first); the code parts, small deviations,
// in a plain sum added by one TwoSum.  The result is the sum of what the
// writers stored to within the final rounding of the (hi, lo) pair, so the
// one rounding of each decoded value (which the collision uses) never
// enters mass.  get(a, wr, wq) returns the parts.
template <int D, class Get>
__device__ __forceinline__ void phi_sum_shifted(const Get& get, float& hi, float& lo)
{
    constexpr int Q = Lat<D>::Q;
    constexpr int C = Q / 2;
    float wr, wq, wr2, wq2;
    get(C, wr, wq);
    float2 h = f2(wr, 0.f), l = f2(0.f, 0.f), q = f2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        const int a = by_weight<D>(k);
        get(a, wr, wq);
        get(Q - 1 - a, wr2, wq2);
        const float2 v = f2(wr, wr2);
        const float2 s = add2(h, v);
        l = add2(l, add2(v, neg2(add2(s, neg2(h)))));
        h = s;
        q = add2(q, f2(wq, wq2));
    }
    // join the reference lanes (TwoSum), add the code sum (TwoSum), renormalise
    float t = h.x + h.y;
    float bb = t - h.x;
    float e = (h.x - (t - bb)) + (h.y - bb);
    const float qs = q.x + q.y;
    const float t2 = t + qs;
    bb = t2 - t;
    e += (t - (t2 - bb)) + (qs - bb);
    const float lsum = (l.x + l.y) + e;
    hi = t2 + lsum;
    lo = lsum - (hi - t2);
}

// R = (th + tl - sq) / den with the subtraction error-free (TwoSum), so that
// the decoded values of a cell add up to its total to within the roundings
// of one addition and one division
template <int D>
__device__ __forceinline__ float ref_from_total(float th, float tl, float sq)
{
    const float d = th - sq;
    const float bb = d - th;
    const float e = (th - (d - bb)) + (-sq - bb);
    return (d + (e + tl)) / wden<D>();
}

// Encoder of one cell's post-collision values: the moving directions in the
// order the collision emits them, then finish(th, tl) with the cell's
// conserved total th + tl in place of the rest value.  off = S v_C/W_C is
// the cell's rest ratio (the rest value from its formula); sq accumulates
// s sum_a W_a q_a (exact products, small terms).
// Seed of the stochastic rounding of the codes a cell writes in one step
// (set 0: f', 1: g): a 32-bit integer hash (two xor-shift-multiply rounds,
// Wellons' lowbias32 constants) of the cell index, the set and the step,
// so that every kernel writing the cell draws the same bits.
__device__ __forceinline__ unsigned mix32(unsigned h)
{
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    h *= 0x846ca68bu;
    h ^= h >> 16;
    return h;
}
__device__ __forceinline__ unsigned code_seed(const DevParams& p, long long cell, int set)
{
    return mix32((unsigned)cell * 2u + (unsigned)set + mix32(p.step));
}
// the code of deviation q for direction a: round to nearest, or
// stochastically with 16 bits drawn from the cell's (fully mixed) seed and a
// by one odd multiplication (the high half of (seed ^ a K1) K2)
template <class St>
__device__ __forceinline__ unsigned short enc_code(float q, unsigned seed, int a)
{
    if constexpr (St::stochastic)
        return St::enc_sr(q, ((seed ^ ((unsigned)a * 0x9e3779b9u)) * 0x85ebca6bu) >> 16);
    else
        return St::enc(q);
}

template <int D, class St>
struct EncSoA {  // cell i of a Pop: R at base + i, codes at stride N
    static constexpr bool kTotal = true;
    float* R;
    unsigned short* q;
    long long N;
    float off;
    mutable float sq;
    unsigned seed;  // code_seed of the writer cell (stochastic rounding)
    __device__ __forceinline__ void operator()(int a, float v) const
    {
        constexpr int C = Lat<D>::Q / 2;
        const float W = wint<D>(a);
        const unsigned short c = enc_code<St>(fmaf(v, St::S / W, -off), seed, a);
        q[(a - (a > C)) * N] = c;
        sq += St::dec(c) * (W * St::s);
    }
    __device__ __forceinline__ void finish(float th, float tl) const { *R = ref_from_total<D>(th, tl, sq); }
};
template <int D, class St>
struct EncPtr {  // per-direction code arrays (entry C unused), one cell index
    static constexpr bool kTotal = true;
    unsigned short* const* qb;
    float* R;
    int self;
    float off;
    mutable float sq;
    unsigned seed;  // code_seed of the writer cell (stochastic rounding)
    __device__ __forceinline__ void operator()(int a, float v) const
    {
        const float W = wint<D>(a);
        const unsigned short c = enc_code<St>(fmaf(v, St::S / W, -off), seed, a);
        qb[a][self] = c;
        sq += St::dec(c) * (W * St::s);
    }
    __device__ __forceinline__ void finish(float th, float tl) const { R[self] = ref_from_total<D>(th, tl, sq); }
};

// Neighbour of the phi stencil: periodic wrap, or the mirrored ghost at a
// wall (the ghost equals the wall cell, reading A17).
__device__ __forceinline__ int wrap_h(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
__device__ __forceinline__ int wrap_v(int v, int n, int periodic)
{
    if (v >= 0 && v < n) return v;
    if (periodic) return v < 0 ? v + n : v - n;
    return v < 0 ? 0 : n - 1;
}
// the same per side of the vertical axis (z-slabs: a wall on one side only)
__device__ __forceinline__ int wrap_vert(const DevParams& p, int v, int n)
{
    if (v >= 0 && v < n) return v;
    if (v < 0) return p.wall_lo ? 0 : v + n;
    return p.wall_hi ? n - 1 : v - n;
}

// ------------------------------------------------------- cells and stencil
__device__ __forceinline__ void cell_xyz(const DevParams& p, long long i, int& x, int& y, int& z)
{
    x = (int)(i % p.nx);
    long long r = i / p.nx;
    y = (int)(r % p.ny);
    z = (int)(r / p.ny);
}

// neighbour index of the phi stencil
template <int D>
__device__ __forceinline__ long long nbr_index(const DevParams& p, int a, int x, int y, int z)
{
    const int xx = wrap_h(x + Lat<D>::cx(a), p.nx);
    if (D == 3) {
        const int yy = wrap_h(y + Lat<D>::cy(a), p.ny);
        const int zz = wrap_vert(p, z + Lat<D>::cz(a), p.nz);
        return ((long long)zz * p.ny + yy) * p.nx + xx;
    } else {
        const int yy = wrap_v(y + Lat<D>::cy(a), p.ny, p.vert_periodic);
        return (long long)yy * p.nx + (p.sym_x ? wrap_v(x + Lat<D>::cx(a), p.nx, 0) : xx);
    }
}

// phi = sum_a g_a (Sec. 2.2) is accumulated as an unevaluated pair hi + lo:
// the stencil below differences neighbouring values of phi, and the chemical
// potential of a near-equilibrium interface is a near-cancelling difference
// of its two terms, so the half-ulp rounding of a plain FP32 sum would
// dominate the FP32 error of the whole step.  The rest population (the
// largest, w = 8/27 or 4/9 of phi) is added first and every later term is
// smaller than the running sum, so Dekker's Fast2Sum recovers each rounding
// error exactly with three additions.
//
// The chain runs as two lanes of paired arithmetic: lane x starts from the
// rest population and takes the directions a < Q/2, lane y starts from zero
// and takes their opposites, both in order of decreasing weight (faces,
// edges, corners) so that each term is no larger than the running sum on
// smooth fields; the lanes are then joined by one TwoSum.

template <int D, class Get>
__device__ __forceinline__ void phi_sum(const Get& get, float& hi, float& lo)
{
    constexpr int Q = Lat<D>::Q;
    constexpr int C = Q / 2;
    float2 h = f2(get(C), 0.f), l = f2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < C; ++k) {
        const int a = by_weight<D>(k);
        const float2 v = f2(get(a), get(Q - 1 - a));
        const float2 s = add2(h, v);
        l = add2(l, add2(v, neg2(add2(s, neg2(h)))));
        h = s;
    }
    // join the lanes exactly, then renormalise (|lo| <= ulp(hi)/2)
    const float t = h.x + h.y;
    const float bb = t - h.x;
    const float e = (h.x - (t - bb)) + (h.y - bb);
    const float lsum = (l.x + l.y) + e;
    hi = t + lsum;
    lo = lsum - (hi - t);
}

// phi of the reduced phase lattice: the rest value, then the face pairs
// (equal weights, so TwoSum rather than Fast2Sum), as a compensated pair
template <int D, class Get>
__device__ __forceinline__ void phi_sum_red(const Get& get, float& hi, float& lo)
{
    constexpr int Q = 2 * D + 1;
    float2 h = f2(get(D), 0.f), l = f2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < D; ++k) two_sum2(h, l, f2(get(k), get(Q - 1 - k)));
    const float t = h.x + h.y;
    const float bb = t - h.x;
    const float e = (h.x - (t - bb)) + (h.y - bb);
    const float lsum = (l.x + l.y) + e;
    hi = t + lsum;
    lo = lsum - (hi - t);
}

template <int D, bool PR, class Get>
__device__ __forceinline__ void phi_sum_phase(const Get& get, float& hi, float& lo)
{
    if constexpr (PR)
        phi_sum_red<D>(get, hi, lo);
    else
        phi_sum<D>(get, hi, lo);
}

// Isotropic differences (Sec. 2.2) from the Q neighbour values
// phi(x + c_a) = nh[a] + nl[a]: grad_i = 3 sum w c_i phi(x+c),
// lap = 6 sum w (phi(x+c) - phi(x)).  Opposite neighbours are taken as a
// pair: the gradient from the difference of their deviations from the
// centre (exactly zero on a uniform field), the Laplacian from their sum.
// nb(a) returns the pair (hi, lo) of phi(x + c_a); centre = nb(C).
template <int D, class NB>
__device__ __forceinline__ void stencil_from(const NB& nb, float2 centre, float grad[3], float& lap)
{
    constexpr int Q = Lat<D>::Q;
    constexpr int C = Q / 2;
    const float2 hc = f2(-centre.x, -centre.x), lc = f2(-centre.y, -centre.y);
    float gx = 0.f, gy = 0.f, gz = 0.f;
    float2 ls = f2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < C; ++a) {
        const int b = Q - 1 - a;
        const float w = Lat<D>::w(a);
        const float2 va = nb(a), vb = nb(b);
        // phi(x + c) - phi(x) and phi(x - c) - phi(x), hi and lo parts differenced first
        const float2 dd = add2(add2(f2(va.x, vb.x), hc), add2(f2(va.y, vb.y), lc));
        ls = fma2(f2(w, w), dd, ls);
        const float d = w * (dd.x - dd.y);
        if (Lat<D>::cx(a)) gx += Lat<D>::cx(a) * d;
        if (Lat<D>::cy(a)) gy += Lat<D>::cy(a) * d;
        if (Lat<D>::cz(a)) gz += Lat<D>::cz(a) * d;
    }
    grad[0] = 3.f * gx;
    grad[1] = 3.f * gy;
    grad[2] = (D == 3) ? 3.f * gz : 0.f;
    lap = 6.f * (ls.x + ls.y);
}

template <int D>
__device__ __forceinline__ void stencil_from_nb(const float* nh, const float* nl, float grad[3], float& lap)
{
    constexpr int C = Lat<D>::Q / 2;
    stencil_from<D>([&](int a) { return f2(nh[a], nl[a]); }, f2(nh[C], nl[C]), grad, lap);
}

// ------------------------------------------------------ flow collision
// Moments of the pre-collision f': P, J, and the second moments Pi_ij.
struct FlowMoments {
    float P, J[3];
    float Pxx, Pyy, Pzz, Pxy, Pxz, Pyz;
};

// Moments of the Q pre-collision values f[a].  J is summed over opposite
// pairs, c_a (f_a - f_opp(a)): the O(w p_h) part common to both members of a
// pair cancels exactly before the sum, so the small momentum of a light phase
// (density ratio up to 1000) is not buried under the pressure in FP32.
template <int D>
__device__ __forceinline__ void flow_moments(FlowMoments& m, const float* f)
{
    constexpr int Q = Lat<D>::Q;
    constexpr int C = Q / 2;
    m.P = f[C];
    m.J[0] = m.J[1] = m.J[2] = 0.f;
    m.Pxx = m.Pyy = m.Pzz = m.Pxy = m.Pxz = m.Pyz = 0.f;
#pragma unroll
    for (int a = 0; a < C; ++a) {
        const int cx = Lat<D>::cx(a), cy = Lat<D>::cy(a), cz = Lat<D>::cz(a);
        const float2 sd = fma2(f2(1.f, -1.f), f2(f[Q - 1 - a], f[Q - 1 - a]), f2(f[a], f[a]));
        const float s = sd.x, d = sd.y;  // f_a + f_opp, f_a - f_opp
        m.P += s;
        if (cx) m.J[0] += cx * d;
        if (cy) m.J[1] += cy * d;
        if (cz) m.J[2] += cz * d;
        if (cx) m.Pxx += s;
        if (cy) m.Pyy += s;
        if (cz) m.Pzz += s;
        if (cx * cy) m.Pxy += (cx * cy) * s;
        if (cx * cz) m.Pxz += (cx * cz) * s;
        if (cy * cz) m.Pyz += (cy * cz) * s;
    }
}

// Per-cell results of the collision set-up that the output loops need.
struct CellState {
    float u[3];        // velocity
    float n[3];        // interface normal
    float rcs2;        // rho cs2
    float ph;          // p_h = P + sum(Xi)/2
    float F[3], uF;    // force density F = F_s + F_b
    float G[3], uG;    // G = cs2 grad(rho)
    float uu;          // |u|^2
    float ew[3][3];    // per-axis product-equilibrium deviation e_d(c) - w1(c), [axis][c+1]
    float phi, sharp;  // phi and lambda_phi 4 phi (1-phi)/W
    float sdiv;        // kFlagDivU: cs2 rho div(u), the zeroth moment of the w cs2 rho div(u) term of Xi
};

// Local closure (Sec. 2.1/2.3; readings A1, A2, A7, A12, A13, A15): density,
// interface normal, chemical potential, force, velocity and p_h of one cell
// into s (every field but ew); returns rho.  Also the observables use it.
// DV (kFlagDivU): Xi keeps its w cs2 rho div(u) term (Sec. 2.3), with divu
// given by the caller; it adds cs2 rho div(u)/2 to p_h.
template <int D, bool DV = false>
__device__ __forceinline__ float flow_closure(const DevParams& p, float phi, const float grad[3], float lap,
                                              const FlowMoments& m, CellState& s, float& inv_rho, float& nu,
                                              float divu = 0.f)
{
    const float rho = p.rho_l + p.drho * phi;
    inv_rho = 1.0f / rho;
    if (p.flags & kFlagDynamicVisc)
        nu = (p.eta_l + (p.eta_h - p.eta_l) * phi) * inv_rho;
    else
        nu = p.nu_h + (p.nu_l - p.nu_h) * (1.0f - phi);
    // interface normal, chemical potential, force
    const float g2 = grad[0] * grad[0] + grad[1] * grad[1] + (D == 3 ? grad[2] * grad[2] : 0.f);
    const float inv_g = 1.0f / fmaxf(sqrtf(g2), 1e-4f);
    const float mu = p.beta2 * phi * (phi - 1.0f) * (2.0f * phi - 1.0f) - p.kappa * lap;
    float F[3];
    F[0] = mu * grad[0];
    F[1] = mu * grad[1];
    F[2] = (D == 3) ? mu * grad[2] : 0.f;
    if (p.flags & kFlagUniformForce)
        F[0] += p.force_x;
    else
        F[D - 1] -= (rho - p.rho_bar) * p.g_accel;

    // u = J/(rho cs2) + F/(2 rho)
    for (int i = 0; i < 3; ++i) {
        s.u[i] = (D == 2 && i == 2) ? 0.f : (3.0f * m.J[i] + 0.5f * F[i]) * inv_rho;
        s.n[i] = (D == 2 && i == 2) ? 0.f : grad[i] * inv_g;
        s.G[i] = (D == 2 && i == 2) ? 0.f : p.drho * grad[i] / 3.0f;
        s.F[i] = F[i];
    }
    const float ux = s.u[0], uy = s.u[1], uz = s.u[2];
    s.uG = ux * s.G[0] + uy * s.G[1] + uz * s.G[2];
    s.uF = ux * F[0] + uy * F[1] + uz * F[2];
    s.uu = ux * ux + uy * uy + uz * uz;
    s.rcs2 = rho / 3.0f;
    s.ph = m.P + 0.5f * s.uG;
    if constexpr (DV) {
        s.sdiv = s.rcs2 * divu;
        s.ph = m.P + 0.5f * (s.uG + s.sdiv);
    }
    s.phi = phi;
    s.sharp = p.lam_sharp * phi * (1.0f - phi);
    return rho;
}

// The relaxation of the flow collision, after the closure (inv_rho and nu
// from flow_closure): the relaxed second-order deviations and the per-axis
// product equilibrium (s.ew).  Produces the 27-entry Kronecker inverse of the
// post-collision moment differences in dh[] (h* - E(u)).
template <int D>
__device__ __forceinline__ void flow_relax(const FlowMoments& m, CellState& s, float inv_rho, float nu, float dh[27])
{
    const float omega = 1.0f / (3.0f * nu + 0.5f);
    const float om1 = 1.0f - omega;
    const float ux = s.u[0], uy = s.u[1], uz = s.u[2];
    float V[3];
    for (int i = 0; i < 3; ++i) V[i] = s.G[i] + s.F[i];
    const float uV = s.uG + s.uF;

    // second moments of f^p minus theta cs2 delta, i.e. with 1/cs2 = 3:
    // [3 Pi_ij - P delta_ij + (u_i V_j + u_j V_i)/2 - 3 u_i u_j u.V/2] / rho - u_i u_j
    // (cs2 itself never enters as a rounded constant)
    const float hV3 = 1.5f * uV;
    float dxx = (3.0f * m.Pxx - m.P + ux * V[0] - ux * ux * hV3) * inv_rho - ux * ux;
    float dyy = (3.0f * m.Pyy - m.P + uy * V[1] - uy * uy * hV3) * inv_rho - uy * uy;
    float dxy = (3.0f * m.Pxy + 0.5f * (ux * V[1] + uy * V[0]) - ux * uy * hV3) * inv_rho - ux * uy;
    float dzz = 0.f, dxz = 0.f, dyz = 0.f;
    if (D == 3) {
        dzz = (3.0f * m.Pzz - m.P + uz * V[2] - uz * uz * hV3) * inv_rho - uz * uz;
        dxz = (3.0f * m.Pxz + 0.5f * (ux * V[2] + uz * V[0]) - ux * uz * hV3) * inv_rho - ux * uz;
        dyz = (3.0f * m.Pyz + 0.5f * (uy * V[2] + uz * V[1]) - uy * uz * hV3) * inv_rho - uy * uz;
    }
    // cumulant relaxation: shear rate on off-diagonal and deviatoric parts,
    // trace to D cs2 (rate one), every higher cumulant to zero (rate one)
    const float tr = (D == 3) ? (dxx + dyy + dzz) * (1.0f / 3.0f) : (dxx + dyy) * 0.5f;
    const float a = om1 * (dxx - tr), b = om1 * (dyy - tr), c = (D == 3) ? om1 * (dzz - tr) : 0.f;
    const float pq = om1 * dxy, qq = om1 * dxz, rr = om1 * dyz;

    // per-axis product equilibrium and its deviation from w1
    for (int i = 0; i < 3; ++i) {
        const float ui = s.u[i], u2 = ui * ui;
        s.ew[i][0] = 0.5f * (u2 - ui);
        s.ew[i][1] = -u2;
        s.ew[i][2] = 0.5f * (u2 + ui);
    }

    // post-collision central-moment differences (Gaussian closure minus the
    // Gaussian of cs2 I), index ia + 3 ib + 9 ic
    float k[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) k[i] = 0.f;
    const float cs2 = kCs2;
    k[2] = a;            // 200
    k[6] = b;            // 020
    k[4] = pq;           // 110
    k[8] = cs2 * (a + b) + a * b + 2.f * pq * pq;  // 220
    if (D == 3) {
        k[18] = c;       // 002
        k[10] = qq;      // 101
        k[12] = rr;      // 011
        k[20] = cs2 * (a + c) + a * c + 2.f * qq * qq;           // 202
        k[24] = cs2 * (b + c) + b * c + 2.f * rr * rr;           // 022
        k[14] = (cs2 + a) * rr + 2.f * pq * qq;                  // 211
        k[16] = (cs2 + b) * qq + 2.f * pq * rr;                  // 121
        k[22] = (cs2 + c) * pq + 2.f * qq * rr;                  // 112
        k[26] = cs2 * cs2 * (a + b + c) + cs2 * (a * b + b * c + c * a) + a * b * c +
                2.f * ((cs2 + a) * rr * rr + (cs2 + b) * qq * qq + (cs2 + c) * pq * pq) + 8.f * pq * qq * rr;  // 222
    }
    // Kronecker inverse about u: per axis (k0,k1,k2) -> (c=-1, 0, +1)
    // m1 = k1 + u k0, m2 = k2 + 2u k1 + u^2 k0; f(0) = k0 - m2, f(+-1) = (m2 +- m1)/2
    constexpr int NZ = (D == 3) ? 3 : 1;
#pragma unroll
    for (int ic = 0; ic < NZ; ++ic)
#pragma unroll
        for (int ib = 0; ib < 3; ++ib) {
            const int o = 3 * ib + 9 * ic;
            const float k0 = k[o], k1 = k[o + 1], k2 = k[o + 2];
            const float m1 = k1 + ux * k0, m2 = k2 + 2.f * ux * k1 + ux * ux * k0;
            k[o] = 0.5f * (m2 - m1);
            k[o + 1] = k0 - m2;
            k[o + 2] = 0.5f * (m2 + m1);
        }
#pragma unroll
    for (int ic = 0; ic < NZ; ++ic)
#pragma unroll
        for (int ia = 0; ia < 3; ++ia) {
            const int o = ia + 9 * ic;
            const float k0 = k[o], k1 = k[o + 3], k2 = k[o + 6];
            const float m1 = k1 + uy * k0, m2 = k2 + 2.f * uy * k1 + uy * uy * k0;
            k[o] = 0.5f * (m2 - m1);
            k[o + 3] = k0 - m2;
            k[o + 6] = 0.5f * (m2 + m1);
        }
    if (D == 3) {
#pragma unroll
        for (int ib = 0; ib < 3; ++ib)
#pragma unroll
            for (int ia = 0; ia < 3; ++ia) {
                const int o = ia + 3 * ib;
                const float k0 = k[o], k1 = k[o + 9], k2 = k[o + 18];
                const float m1 = k1 + uz * k0, m2 = k2 + 2.f * uz * k1 + uz * uz * k0;
                k[o] = 0.5f * (m2 - m1);
                k[o + 9] = k0 - m2;
                k[o + 18] = 0.5f * (m2 + m1);
            }
    }
#pragma unroll
    for (int i = 0; i < 27; ++i) dh[i] = k[i];
}

// The closure and the relaxation of one cell: s (every field) and dh[].
template <int D, bool DV = false>
__device__ __forceinline__ void flow_collide(const DevParams& p, float phi, const float grad[3], float lap,
                                             const FlowMoments& m, CellState& s, float dh[27], float divu = 0.f)
{
    float inv_rho, nu;
    flow_closure<D, DV>(p, phi, grad, lap, m, s, inv_rho, nu, divu);
    flow_relax<D>(m, s, inv_rho, nu, dh);
}

// Deviation of the second-order Hermite equilibrium f_eq/rho (App. A) from
// its rest value: Gamma_a - w_a = w_a [c.u/cs2 + ((c.u)^2 - cs2 u^2)/(2 cs4)].
template <int D>
__device__ __forceinline__ float gamma_dev(const CellState& s, int a)
{
    const int cx = Lat<D>::cx(a), cy = Lat<D>::cy(a), cz = Lat<D>::cz(a);
    const float cu = cx * s.u[0] + cy * s.u[1] + cz * s.u[2];
    return Lat<D>::w(a) * (3.0f * cu + 4.5f * cu * cu - 1.5f * s.uu);
}

// Post-collision f'*_a = rho cs2 (h*_a - w_a) + w_a p_h + Xi_a/2 with
// h* - w = (E(u) - w) + dh and the source (Sec. 2.3, reading A6)
//   Xi_a = cs2 (Gamma_a - w_a)(c_a - u).grad(rho) + Gamma_a (c_a - u).F,
// both terms formed from small factors (no O(w |grad rho|) cancellation).
template <int D>
__device__ __forceinline__ float flow_post(const CellState& s, const float dh[27], int a, float gdev)
{
    const int cx = Lat<D>::cx(a), cy = Lat<D>::cy(a), cz = Lat<D>::cz(a);
    const float w = Lat<D>::w(a);
    const float cG = cx * s.G[0] + cy * s.G[1] + cz * s.G[2] - s.uG;
    const float cF = cx * s.F[0] + cy * s.F[1] + cz * s.F[2] - s.uF;
    const float xi = gdev * cG + (w + gdev) * cF;
    // telescoped E - w = e_x e_y e_z - w_x w_y w_z
    const float wy = (float)w1d(cy), wz = (float)w1d(cz);
    const float ex = (float)w1d(cx) + s.ew[0][cx + 1], ey = wy + s.ew[1][cy + 1];
    float ew;
    if (D == 3)
        ew = s.ew[0][cx + 1] * wy * wz + ex * s.ew[1][cy + 1] * wz + ex * ey * s.ew[2][cz + 1];
    else
        ew = s.ew[0][cx + 1] * wy + ex * s.ew[1][cy + 1];
    return s.rcs2 * (ew + dh[a]) + w * s.ph + 0.5f * xi;
}

// Phase-field BGK with the sharpening source (Sec. 2.2, readings A3-A5):
// g* = g + (phi Gamma - g)/tau + lambda w (c.n) 4 phi (1-phi)/W
template <int D>
__device__ __forceinline__ float phase_post(const DevParams& p, const CellState& s, int a, float g, float gdev)
{
    const int cx = Lat<D>::cx(a), cy = Lat<D>::cy(a), cz = Lat<D>::cz(a);
    const float w = Lat<D>::w(a);
    const float cn = cx * s.n[0] + cy * s.n[1] + cz * s.n[2];
    return g + p.inv_tau_phi * (s.phi * (w + gdev) - g) + w * cn * s.sharp;
}

// Offsets S v_C/W_C of the shifted encoders: the rest populations of f' and
// g from their formulas (the rest value emitted last equals them to within
// rounding).
template <int D, class St, class GSrc>
__device__ __forceinline__ void rest_offsets(const DevParams& p, const CellState& s, const float dh[27],
                                             const GSrc& gin, float& off_f, float& off_g)
{
    constexpr int C = Lat<D>::Q / 2;
    const float gd = gamma_dev<D>(s, C);
    const float k = St::S / wint<D>(C);
    off_f = k * flow_post<D>(s, dh, C, gd);
    off_g = k * phase_post<D>(p, s, C, gin(C), gd);
}

// All post-collision populations of one cell.  The moving populations follow
// the formulas above; the rest population (a = Q/2) is formed last from the
// exact conservation identities of the collision,
//   sum_a g*_a = sum_a g_a                     (sum S_bar = 0, sum g_eq = phi)
//   sum_a f'*_a = sum_a f'_a + cs2 u.grad(rho)  (sum Xi = cs2 u.grad(rho)),
// so that the FP32 rounding of the weights (their float values sum to
// 1 + 7.45e-9) cannot bias mass or pressure step after step; what remains
// is unbiased round-off.  In exact arithmetic this is the value of the formula.
// Sources of the pre-collision g (register array, or a strided shared-memory
// column) and destinations of the post-collision values (strided SoA).
struct GFromArray {
    const float* v;
    __device__ __forceinline__ float operator()(int a) const { return v[a]; }
};
struct GFromStrided {
    const float* base;
    int stride;
    __device__ __forceinline__ float operator()(int a) const { return base[a * stride]; }
};
struct PtrOut {  // per-direction array bases, one cell index
    static constexpr bool kTotal = false;
    float* const* base;
    int self;
    __device__ __forceinline__ void operator()(int a, float v) const { base[a][self] = v; }
};
struct SoAOut {
    static constexpr bool kTotal = false;
    float* base;
    long long stride;
    __device__ __forceinline__ void operator()(int a, float v) const { base[a * stride] = v; }
};

// The outputs are formed for each direction a together with its opposite
// (c -> -c, same weight): (a, opp(a)) are the two lanes of the paired FP32
// arithmetic, and the shared factors (c.u, (c.u)^2, c.G, c.F, c.n) are
// computed once per pair.
// dh source: the register array of flow_collide, or a copy parked in shared
// memory (strided per thread) to lower register pressure in the output loop
struct DhArray {
    const float* v;
    __device__ __forceinline__ float operator[](int a) const { return v[a]; }
};
struct DhStrided {
    const float* base;
    int stride;
    __device__ __forceinline__ float operator[](int a) const { return base[a * stride]; }
};

// Reduced phase lattice: d/dt(phi u) of cell i as the backward difference
// phi u - (phi u of the previous step), and this step's phi u stored in its
// place ([k][cell]; each cell reads and writes only its own entries).
template <int D>
__device__ __forceinline__ void phiu_step(const DevParams& p, const CellState& s, float* __restrict__ phiu,
                                          long long i, float d[3])
{
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const float v = s.phi * s.u[k];
        d[k] = v - phiu[k * p.N + i];
        phiu[k * p.N + i] = v;
    }
    if (D == 2) d[2] = 0.f;
}

// Source of d/dt(phi u) for collide_outputs: phiu_step on the stored array
// (called once, after the flow outputs, so its values are not live across
// them), or none on the full phase lattice.
template <int D>
struct PhiUStep {
    const DevParams& p;
    float* phiu;
    long long i;
    __device__ __forceinline__ void operator()(const CellState& s, float d[3]) const { phiu_step<D>(p, s, phiu, i, d); }
};
// the same with the previous value already staged in shared memory
// (prev[k * stride]); the new value goes to the stored array
template <int D>
struct PhiUStaged {
    const DevParams& p;
    float* phiu;
    long long i;
    const float* prev;
    int stride;
    __device__ __forceinline__ void operator()(const CellState& s, float d[3]) const
    {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const float v = s.phi * s.u[k];
            d[k] = v - prev[k * stride];
            phiu[k * p.N + i] = v;
        }
        if (D == 2) d[2] = 0.f;
    }
};
struct NoPhiU {
    __device__ __forceinline__ void operator()(const CellState&, float d[3]) const { d[0] = d[1] = d[2] = 0.f; }
};

// Per-pair pieces of the outputs.  Direction a < Q/2 and its opposite
// b = Q-1-a are the two lanes (c, -c) of the paired arithmetic.
//
// pair_gamma: the equilibrium deviation Gamma - w = w [3 c.u + 4.5 (c.u)^2 -
// 1.5 u^2] (gd) and Gamma itself (wgd = w + gd); m15uu = -1.5 |u|^2.
template <int D>
__device__ __forceinline__ void pair_gamma(const CellState& s, int a, float m15uu, float2& gd, float2& wgd)
{
    const int cx = Lat<D>::cx(a), cy = Lat<D>::cy(a), cz = Lat<D>::cz(a);
    const float w = Lat<D>::w(a);
    const float2 w2 = f2(w, w);
    const float cu = cx * s.u[0] + cy * s.u[1] + cz * s.u[2];
    const float X = fmaf(4.5f * cu, cu, m15uu);
    gd = mul2(w2, fma2(f2(3.f, -3.f), f2(cu, cu), f2(X, X)));
    wgd = add2(w2, gd);
}

// pair_flow: f'* = rho cs2 (E - w + dh) + w p_h + Xi/2 of the pair, with
// Xi = (Gamma - w)(c - u).G + Gamma (c - u).F and E(u) - w telescoped over
// the axes; dab = (dh[a], dh[b]).
template <int D, bool DV>
__device__ __forceinline__ float2 pair_flow(const CellState& s, int a, float2 gd, float2 wgd, float2 dab)
{
    const int cx = Lat<D>::cx(a), cy = Lat<D>::cy(a), cz = Lat<D>::cz(a);
    const float w = Lat<D>::w(a);
    const float2 pm1 = f2(1.f, -1.f);
    const float cG0 = cx * s.G[0] + cy * s.G[1] + cz * s.G[2];
    const float cF0 = cx * s.F[0] + cy * s.F[1] + cz * s.F[2];
    const float2 cG = fma2(pm1, f2(cG0, cG0), f2(-s.uG, -s.uG));
    const float2 cF = fma2(pm1, f2(cF0, cF0), f2(-s.uF, -s.uF));
    float2 xi = fma2(gd, cG, mul2(wgd, cF));
    if constexpr (DV) xi = add2(xi, f2(w * s.sdiv, w * s.sdiv));
    const float2 exs = f2(s.ew[0][cx + 1], s.ew[0][1 - cx]);
    const float2 eys = f2(s.ew[1][cy + 1], s.ew[1][1 - cy]);
    const float wx = (float)w1d(cx), wy = (float)w1d(cy), wz = (float)w1d(cz);
    const float2 ex = add2(f2(wx, wx), exs);
    float2 ew;
    if (D == 3) {
        const float2 ezs = f2(s.ew[2][cz + 1], s.ew[2][1 - cz]);
        const float2 ey = add2(f2(wy, wy), eys);
        ew = fma2(mul2(ex, ey), ezs, fma2(mul2(ex, eys), f2(wz, wz), mul2(exs, f2(wy * wz, wy * wz))));
    } else {
        ew = fma2(ex, eys, mul2(exs, f2(wy, wy)));
    }
    const float wph = w * s.ph;
    return fma2(f2(s.rcs2, s.rcs2), add2(ew, dab), fma2(f2(0.5f, 0.5f), xi, f2(wph, wph)));
}

// pair_phase: g* = g + (phi Gamma - g)/tau + w (c.n) lambda 4 phi (1-phi)/W
// of the pair (flow lattice), gi = (g_a, g_b) pre-collision
template <int D>
__device__ __forceinline__ float2 pair_phase(const DevParams& p, const CellState& s, int a, float2 wgd, float2 gi)
{
    const int cx = Lat<D>::cx(a), cy = Lat<D>::cy(a), cz = Lat<D>::cz(a);
    const float w = Lat<D>::w(a);
    const float2 pm1 = f2(1.f, -1.f);
    const float cn0 = cx * s.n[0] + cy * s.n[1] + cz * s.n[2];
    const float ws = w * s.sharp;
    const float2 itau = f2(p.inv_tau_phi, p.inv_tau_phi);
    return fma2(f2(ws, ws), mul2(pm1, f2(cn0, cn0)), fma2(itau, fma2(f2(s.phi, s.phi), wgd, neg2(gi)), gi));
}

// The rest populations from the conservation identities (see below): the
// flow total P + u.G (+ the divergence term) less the moving outputs fs,
// the phase-field total (gsum_hi, gsum_lo) less the compensated moving
// outputs (gs, gl); or a shifted encoder takes the totals themselves.
template <bool DV, class Out>
__device__ __forceinline__ void flow_rest(const CellState& s, const FlowMoments& m, float2 fs, const Out& fout,
                                          int C)
{
    if constexpr (Out::kTotal)
        fout.finish(m.P, s.uG);
    else
        fout(C, (DV ? (m.P + s.uG) + s.sdiv : m.P + s.uG) - (fs.x + fs.y));
}
template <class Out>
__device__ __forceinline__ void phase_rest(float gsum_hi, float gsum_lo, float2 gs, float2 gl, const Out& gout, int GC)
{
    if constexpr (Out::kTotal) {
        gout.finish(gsum_hi, gsum_lo);
    } else {
        float t = gs.x + gs.y;  // combine the lanes exactly
        const float bb = t - gs.x;
        const float e = (gs.x - (t - bb)) + (gs.y - bb);
        gout(GC, (gsum_hi - t) + (gsum_lo - (gl.x + gl.y + e)));
    }
}

// The phase-field update on the reduced lattice: g* = g + (g_eq - g)/tau +
// w c.(lambda 4 phi(1-phi)/W n + lambda/cs2 d/dt(phi u)) with the
// first-order equilibrium g_eq = w phi (1 + c.u/cs2), the sharpening source
// and the correction term (Sec. 2.2), lanes (r, opposite); the rest slot
// from the conserved total.
template <int D, class GSrc, class Out, class DPhiU>
__device__ __forceinline__ void phase_outputs_reduced(const DevParams& p, const CellState& s, const GSrc& gin,
                                                      float gsum_hi, float gsum_lo, const Out& gout,
                                                      const DPhiU& dphiu_fn, float2 gs, float2 gl)
{
    constexpr int GC = PhaseLat<D, true>::C;
    constexpr float ics = PhaseLat<D, true>::inv_cs2;
    const float2 itau = f2(p.inv_tau_phi, p.inv_tau_phi);
    const float2 pm1 = f2(1.f, -1.f);
    float qv[3];
    dphiu_fn(s, qv);
#pragma unroll
    for (int i = 0; i < 3; ++i) qv[i] = fmaf(p.lam_corr, qv[i], s.sharp * s.n[i]);
#pragma unroll
    for (int r = 0; r < GC; ++r) {
        const int a = PhaseLat<D, true>::full(r);
        const int cx = Lat<D>::cx(a), cy = Lat<D>::cy(a), cz = Lat<D>::cz(a);
        const float w = PhaseLat<D, true>::w(r);
        const float cu = cx * s.u[0] + cy * s.u[1] + cz * s.u[2];
        const float cq = cx * qv[0] + cy * qv[1] + cz * qv[2];
        const float wphi = w * s.phi;
        const float t = wphi * ics * cu;
        const float2 geq = fma2(pm1, f2(t, t), f2(wphi, wphi));
        const float2 gi = f2(gin(r), gin(2 * GC - r));
        const float2 go = fma2(f2(w, w), mul2(pm1, f2(cq, cq)), fma2(itau, add2(geq, neg2(gi)), gi));
        gout(r, go.x);
        gout(2 * GC - r, go.y);
        two_sum2(gs, gl, go);
    }
    phase_rest(gsum_hi, gsum_lo, gs, gl, gout, GC);
}

// PR: g on the reduced phase lattice (gin / gout index its slots), with
// dphiu(s, d) giving d/dt(phi u) of the cell for the correction term.
// DV: the w cs2 rho div(u) term of Xi (s.sdiv from flow_closure<D, true>):
// half of it reaches f'* through p_h, half through Xi/2.
template <int D, bool PR = false, bool DV = false, class GSrc, class Out, class DH, class DPhiU = NoPhiU>
__device__ __forceinline__ void collide_outputs(const DevParams& p, const CellState& s, const DH& dh,
                                                const FlowMoments& m, const GSrc& gin, float gsum_hi,
                                                float gsum_lo, const Out& fout, const Out& gout,
                                                const DPhiU& dphiu_fn = DPhiU{})
{
    static_assert(!(PR && Out::kTotal), "the reduced phase lattice is stored in FP32 only");
    static_assert(!(DV && Out::kTotal), "the divergence term is supported with FP32 storage only");
    constexpr int Q = Lat<D>::Q;
    constexpr int C = Q / 2;
    const float m15uu = -1.5f * s.uu;
    float2 fs = f2(0.f, 0.f), gs = f2(0.f, 0.f), gl = f2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < C; ++a) {
        const int b = Q - 1 - a;
        float2 gd, wgd;
        pair_gamma<D>(s, a, m15uu, gd, wgd);
        const float2 fo = pair_flow<D, DV>(s, a, gd, wgd, f2(dh[a], dh[b]));
        fout(a, fo.x);
        fout(b, fo.y);
        fs = add2(fs, fo);
        if constexpr (!PR) {
            const float2 go = pair_phase<D>(p, s, a, wgd, f2(gin(a), gin(b)));
            gout(a, go.x);
            gout(b, go.y);
            two_sum2(gs, gl, go);
        }
    }
    // target totals: P + u.G (flow) and the incoming sum (phase field); the
    // rest populations take the difference (conservation identities above),
    // or a shifted encoder takes the totals themselves
    flow_rest<DV>(s, m, fs, fout, C);
    if constexpr (PR)
        phase_outputs_reduced<D>(p, s, gin, gsum_hi, gsum_lo, gout, dphiu_fn, gs, gl);
    else
        phase_rest(gsum_hi, gsum_lo, gs, gl, gout, C);
}

// The same outputs in two passes, phase field first: phase_outputs needs only
// the closure (CellState without ew), so a kernel can run it before
// flow_relax and reuse the staged pre-collision g for the moment
// differences; flow_outputs then emits f'.  Each value is formed by the same
// operations as in collide_outputs, and the rest populations accumulate the
// moving ones in the same order, so the results are identical.
template <int D, class GSrc, class Out>
__device__ __forceinline__ void phase_outputs(const DevParams& p, const CellState& s, const GSrc& gin, float gsum_hi,
                                              float gsum_lo, const Out& gout)
{
    constexpr int Q = Lat<D>::Q;
    constexpr int C = Q / 2;
    const float m15uu = -1.5f * s.uu;
    float2 gs = f2(0.f, 0.f), gl = f2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < C; ++a) {
        const int b = Q - 1 - a;
        float2 gd, wgd;
        pair_gamma<D>(s, a, m15uu, gd, wgd);
        const float2 go = pair_phase<D>(p, s, a, wgd, f2(gin(a), gin(b)));
        gout(a, go.x);
        gout(b, go.y);
        two_sum2(gs, gl, go);
        out_pair_done();
    }
    phase_rest(gsum_hi, gsum_lo, gs, gl, gout, C);
}
template <int D, class Out, class DH>
__device__ __forceinline__ void flow_outputs(const CellState& s, const DH& dh, const FlowMoments& m, const Out& fout)
{
    constexpr int Q = Lat<D>::Q;
    constexpr int C = Q / 2;
    const float m15uu = -1.5f * s.uu;
    float2 fs = f2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < C; ++a) {
        const int b = Q - 1 - a;
        float2 gd, wgd;
        pair_gamma<D>(s, a, m15uu, gd, wgd);
        const float2 fo = pair_flow<D, false>(s, a, gd, wgd, f2(dh[a], dh[b]));
        fout(a, fo.x);
        fout(b, fo.y);
        fs = add2(fs, fo);
        out_pair_done();
    }
    flow_rest<false>(s, m, fs, fout, C);
}

}  // namespace lbmp
