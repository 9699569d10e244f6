// lbmp_tile.cuh -- tile geometry and staging helpers of the fused D3Q27
// step kernels (FP32 and shifted 16-bit storage forms).
#pragma once

#include <type_traits>

#include "lbmp_internal.h"

// The tile shape is fixed per translation unit (LBMP_FUSED_TX / _TY); a unit
// that builds another shape names its own namespace (LBMP_TILE_NS).
#ifndef LBMP_TILE_NS
#define LBMP_TILE_NS tile
#endif

namespace lbmp {
namespace LBMP_TILE_NS {

// tile shape and CTAs per SM (compile-time; the defaults are the measured best)
#ifndef LBMP_FUSED_TX
#define LBMP_FUSED_TX 32
#endif
#ifndef LBMP_FUSED_TY
#define LBMP_FUSED_TY 4
#endif
#ifndef LBMP_FUSED_MINB
#define LBMP_FUSED_MINB 3
#endif
// 1: f' of the plane is staged by cp.async into shared memory with the g
// copies (frees the registers of 27 loads in flight); 0: loaded to registers
#ifndef LBMP_FUSED_FSMEM
#define LBMP_FUSED_FSMEM 0
#endif
// 1: the 27 post-collision moment differences are parked in shared memory
// between the collision set-up and the output loop
#ifndef LBMP_FUSED_DHSMEM
#define LBMP_FUSED_DHSMEM 1
#endif
// 1: the phase field on the reduced lattice D3Q7 (LBMP_FLAG_PHASE_REDUCED)
#ifndef LBMP_PHASE_REDUCED
#define LBMP_PHASE_REDUCED 0
#endif
// 1 (full phase lattice only): the phase-field outputs are emitted first, so
// the staged pre-collision g of the plane is consumed before the flow
// relaxation, which then parks its 27 moment differences in that g column
// (no separate shared-memory array for them)
#ifndef LBMP_FUSED_SPLIT
#define LBMP_FUSED_SPLIT 0
#endif
// 1: the ring cells' g are loaded to registers and summed at once by the
// ring threads (no shared-memory ring buffer)
#ifndef LBMP_FUSED_RINGREG
#define LBMP_FUSED_RINGREG 0
#endif
// E > 0: the column and plane offsets are unsigned byte offsets of E-byte
// populations, so a pulled value's address is its array base plus one
// 32-bit sum (every array below 4 GiB); 0: signed element indices, scaled
// to a 64-bit offset at every access
#ifndef LBMP_FUSED_BYTEOFF
#define LBMP_FUSED_BYTEOFF 0
#endif
#if LBMP_FUSED_BYTEOFF
using cell_off = unsigned;
constexpr unsigned kOffUnit = LBMP_FUSED_BYTEOFF;
#else
using cell_off = int;
constexpr int kOffUnit = 1;
#endif
constexpr int TX = LBMP_FUSED_TX, TY = LBMP_FUSED_TY, NT = TX * TY;
constexpr int RX = TX + 2, RY = TY + 2;
constexpr int PLANE = RY * RX;
constexpr int NRING = 2 * RX + 2 * TY;
constexpr int Q3 = 27;
constexpr bool PR = LBMP_PHASE_REDUCED != 0;
constexpr int QG = PhaseLat<3, PR>::Q;  // phase-field populations
constexpr bool kSplit = LBMP_FUSED_SPLIT != 0 && !PR;
constexpr bool kRingReg = LBMP_FUSED_RINGREG != 0;
constexpr bool kDhSmem = LBMP_FUSED_DHSMEM != 0 && !kSplit;
constexpr size_t kSmemBytes =
    sizeof(float) * ((2 * QG + (LBMP_FUSED_FSMEM + (kDhSmem ? 1 : 0)) * Q3) * NT + (kRingReg ? 0 : QG * NRING) +
                     (PR ? 2 * 3 * NT : 0)) +
    sizeof(float2) * 3 * PLANE;
static_assert(NRING <= NT, "one thread per ring cell");

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ int pmod(int v, int n)
{
    const int r = v % n;
    return r < 0 ? r + n : r;
}

// A column (x, y) and its upstream neighbours: xs[c+1] = x - c and
// ys[c+1] = (y - c) nx, wrapped periodically.
struct Column {
    cell_off xs[3], ys[3];
};

__device__ __forceinline__ void set_column(Column& C, const DevParams& p, int x, int y)
{
    C.xs[0] = (cell_off)(x + 1 == p.nx ? 0 : x + 1) * kOffUnit;
    C.xs[1] = (cell_off)x * kOffUnit;
    C.xs[2] = (cell_off)(x == 0 ? p.nx - 1 : x - 1) * kOffUnit;
    C.ys[0] = (cell_off)((y + 1 == p.ny ? 0 : y + 1) * p.nx) * kOffUnit;
    C.ys[1] = (cell_off)(y * p.nx) * kOffUnit;
    C.ys[2] = (cell_off)((y == 0 ? p.ny - 1 : y - 1) * p.nx) * kOffUnit;
}

// element index of a cell offset
__device__ __forceinline__ int elem_index(cell_off o) { return (int)(o / kOffUnit); }

// A plane z and its upstream planes zs[c+1] = (z - c) nx ny; lo/hi flag the
// bottom/top plane of a walled domain, where the population arriving across
// the wall is the opposite population of the cell itself (half-way
// bounce-back).
struct Plane {
    cell_off zs[3];
    bool lo, hi;
};

__device__ __forceinline__ void set_plane(Plane& P, const DevParams& p, int z)
{
    const int nxy = p.nx * p.ny;
    P.lo = p.wall_lo && z == 0;
    P.hi = p.wall_hi && z == p.nz - 1;
    P.zs[0] = (cell_off)((z + 1 == p.nz ? 0 : z + 1) * nxy) * kOffUnit;
    P.zs[1] = (cell_off)(z * nxy) * kOffUnit;
    P.zs[2] = (cell_off)((z == 0 ? p.nz - 1 : z - 1) * nxy) * kOffUnit;
}

// element of an array at cell offset o
template <class E>
__device__ __forceinline__ E* at_cell(E* base, cell_off o)
{
    if constexpr (LBMP_FUSED_BYTEOFF != 0) {
        static_assert(sizeof(E) == kOffUnit, "byte offsets of the unit's population size");
        using B = typename std::conditional<std::is_const<E>::value, const char, char>::type;
        return reinterpret_cast<E*>(reinterpret_cast<B*>(base) + o);
    } else {
        return base + o;
    }
}

// pointer to the post-streaming population a of the cell (column C, plane P);
// Walls = false is the path of every plane that does not touch a wall
template <bool Walls, int a, class E>
__device__ __forceinline__ const E* pulled(const E* const* base, const Column& C, const Plane& P)
{
    constexpr int cx = Lat<3>::cx(a), cy = Lat<3>::cy(a), cz = Lat<3>::cz(a);
    if (Walls && ((cz == 1 && P.lo) || (cz == -1 && P.hi)))
        return at_cell(base[Lat<3>::opp(a)], P.zs[1] + C.ys[1] + C.xs[1]);
    return at_cell(base[a], P.zs[cz + 1] + C.ys[cy + 1] + C.xs[cx + 1]);
}

// compile-time loop over the directions (keeps base[a] a constant-bank operand)
template <int N>
struct Unroll {
    template <class F>
    __device__ __forceinline__ static void run(const F& f)
    {
        Unroll<N - 1>::run(f);
        f.template step<N - 1>();
    }
};
template <>
struct Unroll<0> {
    template <class F>
    __device__ __forceinline__ static void run(const F&)
    {
    }
};

// pointer to the post-streaming phase-field population of slot r (the
// flow-lattice direction PhaseLat::full(r)) of the cell (C, P)
template <bool Walls, int r, class E>
__device__ __forceinline__ const E* pulled_g(const E* const* base, const Column& C, const Plane& P)
{
    constexpr int a = PhaseLat<3, PR>::full(r);
    constexpr int cx = Lat<3>::cx(a), cy = Lat<3>::cy(a), cz = Lat<3>::cz(a);
    if (Walls && ((cz == 1 && P.lo) || (cz == -1 && P.hi))) return at_cell(base[QG - 1 - r], P.zs[1] + C.ys[1] + C.xs[1]);
    return at_cell(base[r], P.zs[cz + 1] + C.ys[cy + 1] + C.xs[cx + 1]);
}

// post-streaming values of the 27 directions of one cell into registers
template <bool Walls>
struct PullLoad {
    const float* const* base;
    const Column& C;
    const Plane& P;
    float* v;
    template <int a>
    __device__ __forceinline__ void step() const
    {
        v[a] = __ldg(pulled<Walls, a>(base, C, P));
    }
};

// post-streaming phase-field values of the QG slots of one cell into registers
template <bool Walls>
struct PullLoadG {
    const float* const* base;
    const Column& C;
    const Plane& P;
    float* v;
    template <int r>
    __device__ __forceinline__ void step() const
    {
        v[r] = __ldg(pulled_g<Walls, r>(base, C, P));
    }
};

// stores of the outputs of one cell (per-direction array bases, one offset)
struct CellOut {
    static constexpr bool kTotal = false;
    float* const* base;
    cell_off self;
    template <class V>  // instantiated only by the units that store through it
    __device__ __forceinline__ void operator()(int a, V v) const
    {
        *at_cell(base[a], self) = v;
    }
};

// plane whose phi stands for plane zz: periodic wrap, or the mirrored ghost
// at a wall (reading A17)
__device__ __forceinline__ int plane_src(const DevParams& p, int zz)
{
    if (zz >= 0 && zz < p.nz) return zz;
    if (zz < 0) return p.wall_lo ? 0 : pmod(zz, p.nz);
    return p.wall_hi ? p.nz - 1 : pmod(zz, p.nz);
}

// per-thread geometry inside a tile: own cell and (for tid < NRING) ring cell
struct ThreadGeo {
    int tid, tx, ty, oslot, lx, ly, rslot;
};

__device__ __forceinline__ ThreadGeo thread_geo()
{
    ThreadGeo T;
    T.tid = threadIdx.x;
    T.tx = T.tid % TX;
    T.ty = T.tid / TX;
    T.oslot = (T.ty + 1) * RX + (T.tx + 1);
    T.lx = T.ly = T.rslot = 0;
    if (T.tid < NRING) {
        const int r = T.tid;
        if (r < RX) {
            T.lx = r - 1;
            T.ly = -1;
        } else if (r < 2 * RX) {
            T.lx = r - RX - 1;
            T.ly = TY;
        } else if (r < 2 * RX + TY) {
            T.lx = -1;
            T.ly = r - 2 * RX;
        } else {
            T.lx = TX;
            T.ly = r - 2 * RX - TY;
        }
        T.rslot = (T.ly + 1) * RX + (T.lx + 1);
    }
    return T;
}

}  // namespace LBMP_TILE_NS
}  // namespace lbmp
