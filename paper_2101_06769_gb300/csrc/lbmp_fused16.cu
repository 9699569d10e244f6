// lbmp_fused16.cu -- the fused D3Q27 step for the shifted 16-bit storage
// forms (FP16 or BF16 codes plus one FP32 reference per cell, layout in
// lbmp_common.cuh).
//
// Work decomposition, summation orders and per-cell arithmetic are those of
// the FP32 fused kernel (lbmp_fused.cu); what differs is the decoding of the
// pulled values and the encoding of the outputs:
//   * a pulled value needs its 16-bit code and the reference R of the cell
//     that wrote it.  The references of the planes around the marching plane
//     are staged in shared memory, four planes per population set in
//     rotation, one new plane per step: g over the tile plus two rings (a ring
//     cell's phi pulls from one cell further out), f' over the tile plus one
//     ring.  Offsets of the staged plane cells are computed once per segment.
//   * cp.async has no 2-byte form, so a g code is copied as the aligned
//     32-bit word that holds it.  nx is even and tile origins are multiples
//     of TX, so the half a thread needs is fixed by its lane parity and the
//     direction's cx (the cell itself for a bounced population), and one byte
//     permute extracts it.
//   * f' codes are loaded to registers (2-byte loads) and decoded after the
//     reference planes are in place.
//   * the ghost plane beyond a wall (mirrored phi, reading A17) is a copy of
//     the wall plane's phi instead of a second staging of that plane.
// the output pair loops keep their memory operations in order (lower register footprint)
#define LBMP_OUT_ORDERED 1
#define LBMP_TILE_NS tile16
#ifndef LBMP_FUSED_BYTEOFF
#define LBMP_FUSED_BYTEOFF 2
#endif
#include <stdint.h>

#include "lbmp_internal.h"
#include "lbmp_tile.cuh"

namespace lbmp {

namespace {

using namespace LBMP_TILE_NS;

// the encoder of one cell's outputs (as EncPtr) at a cell offset of the tile
// geometry: the codes at base + offset, the reference at its 4-byte slot
template <class St>
struct EncCell {
    static constexpr bool kTotal = true;
    unsigned short* const* qb;
    float* R;
    cell_off self;
    float off;
    mutable float sq;
    unsigned seed;  // code_seed of the writer cell (stochastic rounding)
    __device__ __forceinline__ void operator()(int a, float v) const
    {
        const float W = wint<3>(a);
        const unsigned short c = enc_code<St>(fmaf(v, St::S / W, -off), seed, a);
        *at_cell(qb[a], self) = c;
        sq += St::dec(c) * (W * St::s);
    }
    __device__ __forceinline__ void finish(float th, float tl) const
    {
        R[elem_index(self)] = ref_from_total<3>(th, tl, sq);
    }
};

constexpr int C3 = 13;
constexpr int GX = TX + 4, GY = TY + 4, GPLANE = GX * GY;  // g reference plane: tile + two rings
// the moment differences are parked in the consumed g column: no array of their own
constexpr size_t kSmem16 = sizeof(float2) * 3 * PLANE +
                           sizeof(float) * (2 * Q3 * NT + Q3 * NRING + 4 * GPLANE + 4 * PLANE) +
                           sizeof(int) * (GPLANE + PLANE);

struct DirPtrs16 {
    const unsigned short* fin[Q3];  // per-direction code arrays; entry C3 unused
    const unsigned short* gin[Q3];
    unsigned short* fout[Q3];
    unsigned short* gout[Q3];
    const float* rfin;  // references
    const float* rgin;
    float* rfout;
    float* rgout;
};

struct FusedArgs16 {
    int tiles_x, tiles_y, chunk, nitems;
};

__device__ __forceinline__ bool ghost_plane(const DevParams& p, int zz)
{
    return !p.vert_periodic && (zz < 0 || zz >= p.nz);
}

// reference plane k (logical index; periodic wrap) into rotation slot k & 3;
// planes beyond a wall are never read (their populations bounce) and are skipped
__device__ __forceinline__ void load_ref_plane(const DevParams& p, const float* src, int k, float* planes, int size,
                                               const int* off, int tid)
{
    int zk = k;
    if (k < 0 || k >= p.nz) {
        if (!p.vert_periodic) return;
        zk = pmod(k, p.nz);
    }
    const float* base = src + zk * (p.nx * p.ny);
    float* d = planes + ((k + 8) & 3) * size;
    for (int e = tid; e < size; e += NT) cp_async4(d + e, base + off[e]);
}

// aligned 32-bit word holding the code of the pulled g population a
template <bool Walls>
struct StageWord {
    const DirPtrs16& D;
    const Column& C;
    const Plane& P;
    float* buf;
    int stride;
    template <int a>
    __device__ __forceinline__ void step() const
    {
        if constexpr (a != C3) {
            const unsigned short* src = pulled<Walls, a>(D.gin, C, P);
            cp_async4(buf + a * stride, (const float*)((uintptr_t)src & ~(uintptr_t)3));
        }
    }
};

template <bool Walls>
struct CodeLoad {
    const unsigned short* const* base;
    const Column& C;
    const Plane& P;
    unsigned short* q;
    template <int a>
    __device__ __forceinline__ void step() const
    {
        if constexpr (a != C3) q[a] = __ldg(pulled<Walls, a>(base, C, P));
    }
};

// Decode the staged words of one cell and sum phi (hi, lo) from the exact
// parts of the values (phi_sum_shifted); Keep: also store the decoded values
// in place (the tile's own cells, whose values the collision reads; ring
// cells need phi only).  R0 is
// the reference plane of the staged plane, Rm / Rp the planes below / above;
// slot is the cell's index in the reference-plane layout of row length RL;
// selA / selB pick the half of a word for a source of the cell's own / the
// other x parity.
template <bool Walls, class St, bool Keep>
__device__ __forceinline__ void decode_g(const float* Rm, const float* R0, const float* Rp, int slot, int RL,
                                         unsigned selA, unsigned selB, bool lo, bool hi, float* buf, int stride,
                                         float& phi_hi, float& phi_lo)
{
    phi_sum_shifted<3>(
        [&](int a, float& wr, float& wq) {
            const int cx = Lat<3>::cx(a), cy = Lat<3>::cy(a), cz = Lat<3>::cz(a);
            const float W = wint<3>(a);
            if (a == C3) {
                wr = W * R0[slot];
                wq = 0.f;
                if (Keep) buf[a * stride] = wr;
            } else {
                const bool bounced = Walls && ((cz == 1 && lo) || (cz == -1 && hi));
                const float* Rpl = cz == 1 ? Rm : (cz == -1 ? Rp : R0);
                const float R = bounced ? R0[slot] : Rpl[slot - cx - cy * RL];
                const unsigned sel = (cx == 0 || bounced) ? selA : selB;
                const float qv = St::dec_word(__float_as_uint(buf[a * stride]), sel);
                wr = W * R;
                wq = qv * (W * St::s);
                if (Keep) buf[a * stride] = dec_value<3, St>(a, qv, R);  // = wr + wq, rounded once
            }
        },
        phi_hi, phi_lo);
}

template <class St>
struct Seg16 {
    const DevParams& p;
    const DirPtrs16& D;
    const ThreadGeo& T;
    const Column& own;
    const Column& ring;
    float* rS;
    float* RG;
    float* RF;
    const int* offG;
    const int* offF;

    // copies for plane zz: reference planes zz+2 (g) and zz+1 (f'), and the
    // g code words of the tile and ring cells (unless zz is a ghost plane)
    __device__ __forceinline__ void issue(int zz, float* gbuf) const
    {
        const int tid = T.tid;
        load_ref_plane(p, D.rgin, zz + 2, RG, GPLANE, offG, tid);
        load_ref_plane(p, D.rfin, zz + 1, RF, PLANE, offF, tid);
        if (!ghost_plane(p, zz)) {
            Plane P;
            set_plane(P, p, plane_src(p, zz));
            if (P.lo || P.hi) {  // uniform across the CTA
                Unroll<Q3>::run(StageWord<true>{D, own, P, gbuf + tid, NT});
                if (tid < NRING) Unroll<Q3>::run(StageWord<true>{D, ring, P, rS + tid, NRING});
            } else {
                Unroll<Q3>::run(StageWord<false>{D, own, P, gbuf + tid, NT});
                if (tid < NRING) Unroll<Q3>::run(StageWord<false>{D, ring, P, rS + tid, NRING});
            }
        }
        cp_async_commit();
    }

    // wait for the copies; decode plane zz (unless a ghost) and write its phi
    __device__ __forceinline__ void finish(int zz, float* gbuf, float2* phi_plane) const
    {
        cp_async_wait_all();
        if (ghost_plane(p, zz)) return;
        const int pz = plane_src(p, zz);
        const bool lo = !p.vert_periodic && pz == 0, hi = !p.vert_periodic && pz == p.nz - 1;
        const float* Rm = RG + ((zz + 7) & 3) * GPLANE;
        const float* R0 = RG + ((zz + 8) & 3) * GPLANE;
        const float* Rp = RG + ((zz + 9) & 3) * GPLANE;
        const int tid = T.tid;
        const unsigned oA = (T.tx & 1) ? St::kSelHi : St::kSelLo, oB = (T.tx & 1) ? St::kSelLo : St::kSelHi;
        const int ogs = (T.ty + 2) * GX + T.tx + 2;
        float h, l;
        if (lo || hi) {
            if (tid < NRING) {
                const unsigned rA = (T.lx & 1) ? St::kSelHi : St::kSelLo, rB = (T.lx & 1) ? St::kSelLo : St::kSelHi;
                decode_g<true, St, false>(Rm, R0, Rp, (T.ly + 2) * GX + T.lx + 2, GX, rA, rB, lo, hi, rS + tid, NRING, h,
                                          l);
                phi_plane[T.rslot] = make_float2(h, l);
            }
            decode_g<true, St, true>(Rm, R0, Rp, ogs, GX, oA, oB, lo, hi, gbuf + tid, NT, h, l);
        } else {
            if (tid < NRING) {
                const unsigned rA = (T.lx & 1) ? St::kSelHi : St::kSelLo, rB = (T.lx & 1) ? St::kSelLo : St::kSelHi;
                decode_g<false, St, false>(Rm, R0, Rp, (T.ly + 2) * GX + T.lx + 2, GX, rA, rB, false, false,
                                           rS + tid, NRING, h, l);
                phi_plane[T.rslot] = make_float2(h, l);
            }
            decode_g<false, St, true>(Rm, R0, Rp, ogs, GX, oA, oB, false, false, gbuf + tid, NT, h, l);
        }
        phi_plane[T.oslot] = make_float2(h, l);
    }

    // phi of the ghost plane = phi of the wall plane (each thread copies the
    // slots it wrote itself)
    __device__ __forceinline__ void copy_phi(const float2* from, float2* to) const
    {
        if (T.tid < NRING) to[T.rslot] = from[T.rslot];
        to[T.oslot] = from[T.oslot];
    }

    // decoded f' of plane z from its codes and the reference planes
    template <bool Walls>
    __device__ __forceinline__ void decode_f(int z, bool lo, bool hi, const unsigned short* q, float* fr) const
    {
        const float* Rm = RF + ((z + 7) & 3) * PLANE;
        const float* R0 = RF + ((z + 8) & 3) * PLANE;
        const float* Rp = RF + ((z + 9) & 3) * PLANE;
        const int o = T.oslot;
#pragma unroll
        for (int a = 0; a < Q3; ++a) {
            const int cx = Lat<3>::cx(a), cy = Lat<3>::cy(a), cz = Lat<3>::cz(a);
            if (a == C3) {
                fr[a] = wint<3>(C3) * R0[o];
            } else {
                const bool bounced = Walls && ((cz == 1 && lo) || (cz == -1 && hi));
                const float* Rpl = cz == 1 ? Rm : (cz == -1 ? Rp : R0);
                const float R = bounced ? R0[o] : Rpl[o - cx - cy * RX];
                fr[a] = dec_value<3, St>(a, St::dec(q[a]), R);
            }
        }
    }
};

template <class St>
__device__ __forceinline__ void fused_segment16(const DevParams& p, const DirPtrs16& Dp, const ThreadGeo& T,
                                                float* smem, int x0, int y0, int z0, int z1)
{
    float2* phiS = (float2*)smem;                // (hi, lo) [3][PLANE]
    float* gS = (float*)(phiS + 3 * PLANE);      // [2][27][NT] staged words, decoded in place
    float* rS = gS + 2 * Q3 * NT;                // [27][NRING] ring cells
    float* RG = rS + Q3 * NRING;                 // [4][GPLANE] g references
    float* RF = RG + 4 * GPLANE;                 // [4][PLANE] f' references
    int* offG = (int*)(RF + 4 * PLANE);
    int* offF = offG + GPLANE;
    const int tid = T.tid;
    Column own, ring;
    set_column(own, p, pmod(x0 + T.tx, p.nx), pmod(y0 + T.ty, p.ny));
    set_column(ring, p, pmod(x0 + T.lx, p.nx), pmod(y0 + T.ly, p.ny));
    const bool valid = (x0 + T.tx < p.nx) && (y0 + T.ty < p.ny);
    for (int e = tid; e < GPLANE; e += NT)
        offG[e] = pmod(y0 + e / GX - 2, p.ny) * p.nx + pmod(x0 + e % GX - 2, p.nx);
    for (int e = tid; e < PLANE; e += NT) offF[e] = pmod(y0 + e / RX - 1, p.ny) * p.nx + pmod(x0 + e % RX - 1, p.nx);
    __syncthreads();
    const Seg16<St> S{p, Dp, T, own, ring, rS, RG, RF, offG, offF};
    // reference planes needed before the first two stagings
    load_ref_plane(p, Dp.rgin, z0 - 2, RG, GPLANE, offG, tid);
    load_ref_plane(p, Dp.rgin, z0 - 1, RG, GPLANE, offG, tid);
    load_ref_plane(p, Dp.rgin, z0, RG, GPLANE, offG, tid);
    load_ref_plane(p, Dp.rfin, z0 - 1, RF, PLANE, offF, tid);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    int sP = 0, sC = 1, sN = 2;
    S.issue(z0 - 1, gS + Q3 * NT);
    S.finish(z0 - 1, gS + Q3 * NT, phiS + sP * PLANE);
    __syncthreads();
    S.issue(z0, gS);
    S.finish(z0, gS, phiS + sC * PLANE);
    if (ghost_plane(p, z0 - 1)) S.copy_phi(phiS + sC * PLANE, phiS + sP * PLANE);
    __syncthreads();
    for (int z = z0; z < z1; ++z) {
        const int cur = (z - z0) & 1;
        // g(z+1) words and the next reference planes in flight while the f'(z) codes load
        S.issue(z + 1, gS + (cur ^ 1) * Q3 * NT);
        Plane P;
        set_plane(P, p, z);
        unsigned short q[Q3];
        if (P.lo || P.hi)
            Unroll<Q3>::run(CodeLoad<true>{Dp.fin, own, P, q});
        else
            Unroll<Q3>::run(CodeLoad<false>{Dp.fin, own, P, q});
        S.finish(z + 1, gS + (cur ^ 1) * Q3 * NT, phiS + sN * PLANE);
        if (ghost_plane(p, z + 1)) S.copy_phi(phiS + sC * PLANE, phiS + sN * PLANE);
        FlowMoments m;
        {
            float fr[Q3];
            if (P.lo || P.hi)
                S.template decode_f<true>(z, P.lo, P.hi, q, fr);
            else
                S.template decode_f<false>(z, false, false, q, fr);
            flow_moments<3>(m, fr);
        }
        __syncthreads();
        if (valid) {
            float nh[Q3], nl[Q3];
#pragma unroll
            for (int a = 0; a < Q3; ++a) {
                const int cz = Lat<3>::cz(a);
                const float2* pl = phiS + (cz < 0 ? sP : (cz == 0 ? sC : sN)) * PLANE;
                const float2 v = pl[T.oslot + Lat<3>::cy(a) * RX + Lat<3>::cx(a)];
                nh[a] = v.x;
                nl[a] = v.y;
            }
            float grad[3], lap;
            stencil_from_nb<3>(nh, nl, grad, lap);
            CellState s;
            const cell_off self = P.zs[1] + own.ys[1] + own.xs[1];
            float* gcol = gS + cur * Q3 * NT + tid;  // this cell's decoded pre-collision g
            const GFromStrided gin{gcol, NT};
            // g first (it needs only the closure); its decoded column then
            // holds the moment differences for the f' outputs.  The rest
            // offsets of the encoders are those of rest_offsets.
            float inv_rho, nu;
            flow_closure<3>(p, nh[13], grad, lap, m, s, inv_rho, nu);
            const float gd = gamma_dev<3>(s, C3);
            const float kS = St::S / wint<3>(C3);
            const EncCell<St> go{Dp.gout, Dp.rgout, self, kS * phase_post<3>(p, s, C3, gin(C3), gd), 0.f,
                                 code_seed(p, elem_index(self), 1)};
            phase_outputs<3>(p, s, gin, nh[13], nl[13], go);
            float dh[27];
            flow_relax<3>(m, s, inv_rho, nu, dh);
#pragma unroll
            for (int a = 0; a < Q3; ++a) gcol[a * NT] = dh[a];
            const EncCell<St> fo{Dp.fout, Dp.rfout, self, kS * flow_post<3>(s, dh, C3, gd), 0.f,
                                 code_seed(p, elem_index(self), 0)};
            flow_outputs<3>(s, DhStrided{gcol, NT}, m, fo);
        }
        __syncthreads();
        const int t = sP;
        sP = sC;
        sC = sN;
        sN = t;
    }
}

template <class St>
__global__ void __launch_bounds__(NT, LBMP_FUSED_MINB) step_fused3s_kernel(DevParams p, FusedArgs16 A, DirPtrs16 Dp)
{
    extern __shared__ __align__(16) float smem16[];
    const ThreadGeo T = thread_geo();
    for (int item = blockIdx.x; item < A.nitems; item += gridDim.x) {
        const int tile = item % (A.tiles_x * A.tiles_y);
        const int chunk = item / (A.tiles_x * A.tiles_y);
        const int z0 = chunk * A.chunk;
        fused_segment16<St>(p, Dp, T, smem16, (tile % A.tiles_x) * TX, (tile / A.tiles_x) * TY, z0,
                            min(z0 + A.chunk, p.nz));
    }
}

// Batch form (FP16 / BF16 members of a batch): as the FP32 batch kernel, a
// CTA looks up the member of each work item in the device table and stages
// its parameters and direction bases in shared memory.
template <class St>
__global__ void __launch_bounds__(NT, LBMP_FUSED_MINB) step_batch3s_kernel(const BatchDomain* __restrict__ table,
                                                                           int ndom, int nitems)
{
    extern __shared__ __align__(16) float smem16[];
    __shared__ DevParams sp;
    __shared__ DirPtrs16 sd;
    __shared__ int s_dom, s_tx, s_ty, s_chunk, s_begin, s_active;
    const ThreadGeo T = thread_geo();
    int cur = -1;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        __syncthreads();  // every thread has read the previous item's shared values
        if (threadIdx.x == 0) {
            int lo = 0, hi = ndom - 1;  // last member with item_begin <= item
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (table[mid].item_begin <= item)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            s_dom = lo;
        }
        __syncthreads();
        const int d = s_dom;
        if (d != cur) {
            const BatchDomain& B = table[d];
            const int par = B.parity;
            const size_t N = (size_t)B.p.N;
            if (threadIdx.x == 0) {
                sp = B.p;
                s_tx = B.tiles_x;
                s_ty = B.tiles_y;
                s_chunk = B.chunk;
                s_begin = B.item_begin;
                s_active = B.steps_left > 0;
                sd.rfin = B.f[par];
                sd.rgin = B.g[par];
                sd.rfout = B.f[par ^ 1];
                sd.rgout = B.g[par ^ 1];
            }
            for (int k = threadIdx.x; k < 4 * Q3; k += blockDim.x) {
                const int set = k / Q3, a = k % Q3;
                const size_t off = (size_t)(a - (a > C3)) * N;
                unsigned short* base = (unsigned short*)((set == 0 || set == 2 ? B.f : B.g)[set < 2 ? par : par ^ 1] + N);
                unsigned short* q = a != C3 ? base + off : nullptr;
                if (set == 0) sd.fin[a] = q;
                if (set == 1) sd.gin[a] = q;
                if (set == 2) sd.fout[a] = q;
                if (set == 3) sd.gout[a] = q;
            }
            cur = d;
            __syncthreads();
        }
        if (!s_active) continue;  // uniform
        const int local = item - s_begin;
        const int tiles = s_tx * s_ty;
        const int tile = local % tiles;
        const int z0 = (local / tiles) * s_chunk;
        fused_segment16<St>(sp, sd, T, smem16, (tile % s_tx) * TX, (tile / s_tx) * TY, z0, min(z0 + s_chunk, sp.nz));
    }
}

template <class St>
struct BatchCfg16 {
    static int dev, cap;
    static cudaError_t prepare(int device)
    {
        if (dev != device) {
            cudaError_t e = cudaFuncSetAttribute(step_batch3s_kernel<St>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kSmem16);
            if (e != cudaSuccess) return e;
            int per_sm = 0, sms = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_batch3s_kernel<St>, NT, kSmem16);
            if (e != cudaSuccess) return e;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
            if (e != cudaSuccess) return e;
            cap = (per_sm > 0 ? per_sm : 1) * sms;
            dev = device;
        }
        return cudaSuccess;
    }
    static cudaError_t launch(const BatchDomain* table, int ndom, int nitems, int device, cudaStream_t stream)
    {
        if (dev != device) return cudaErrorNotReady;  // prepare first
        if (nitems <= 0) return cudaSuccess;
        const int grid = nitems < cap ? nitems : cap;
        step_batch3s_kernel<St><<<grid, NT, kSmem16, stream>>>(table, ndom, nitems);
        return cudaGetLastError();
    }
};
template <class St>
int BatchCfg16<St>::dev = -1;
template <class St>
int BatchCfg16<St>::cap = 0;

struct Cfg16 {
    int device = -1;
    int per_sm = 0, sms = 0;
};

template <class St>
cudaError_t launch16(lbmp_handle* h, Cfg16& cfg)
{
    if (cfg.device != h->device) {
        cudaError_t e = cudaFuncSetAttribute(step_fused3s_kernel<St>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmem16);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_fused3s_kernel<St>, NT, kSmem16);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
        if (e != cudaSuccess) return e;
        cfg.per_sm = per_sm > 0 ? per_sm : 1;
        cfg.sms = sms;
        cfg.device = h->device;
    }
    DirPtrs16 D;
    const int s = h->parity, d = 1 - h->parity;
    const size_t N = (size_t)h->N;
    const unsigned short* cf = (const unsigned short*)(h->f[s] + N);
    const unsigned short* cg = (const unsigned short*)(h->g[s] + N);
    unsigned short* of = (unsigned short*)(h->f[d] + N);
    unsigned short* og = (unsigned short*)(h->g[d] + N);
    for (int a = 0; a < Q3; ++a) {
        const size_t off = (size_t)(a - (a > C3)) * N;
        const bool mv = a != C3;
        D.fin[a] = mv ? cf + off : nullptr;
        D.gin[a] = mv ? cg + off : nullptr;
        D.fout[a] = mv ? of + off : nullptr;
        D.gout[a] = mv ? og + off : nullptr;
    }
    D.rfin = h->f[s];
    D.rgin = h->g[s];
    D.rfout = h->f[d];
    D.rgout = h->g[d];
    FusedArgs16 A;
    A.tiles_x = (h->grid.nx + TX - 1) / TX;
    A.tiles_y = (h->grid.ny + TY - 1) / TY;
    const LaunchShape L = launch_shape(h, A.tiles_x * A.tiles_y, h->grid.nz, cfg.per_sm, cfg.sms);
    A.chunk = L.chunk;
    A.nitems = L.nitems;
    step_fused3s_kernel<St><<<L.grid, NT, kSmem16, h->stream>>>(h->dp, A, D);
    return cudaGetLastError();
}

Cfg16 g_cfg_f16, g_cfg_bf16;

}  // namespace

const Batch3Ops batch3_ops_f16 = {TX, TY, BatchCfg16<StoreF16>::prepare, BatchCfg16<StoreF16>::launch, nullptr, 0};
const Batch3Ops batch3_ops_bf16 = {TX, TY, BatchCfg16<StoreBF16>::prepare, BatchCfg16<StoreBF16>::launch, nullptr, 0};

cudaError_t launch_step_fused16(lbmp_handle* h)
{
    if (h->D != 3 || (h->grid.nx & 1)) return cudaErrorInvalidValue;
    if (h->params.storage == LBMP_FP16_SHIFTED) return launch16<StoreF16>(h, g_cfg_f16);
    if (h->params.storage == LBMP_BF16_SHIFTED) return launch16<StoreBF16>(h, g_cfg_bf16);
    return cudaErrorInvalidValue;
}

}  // namespace lbmp
