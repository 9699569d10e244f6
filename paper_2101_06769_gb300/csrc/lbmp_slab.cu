// lbmp_slab.cu -- z-slabs (one rank's planes of a D3Q27 domain decomposed
// along z) and the whole-plane copies their exchange uses (include/lbmp.h).
//
// A slab is an ordinary handle whose local grid holds the slab's planes plus
// two ghost planes on every face that borders another slab.  Its vertical
// axis keeps the domain's wall on a face that is the domain's own boundary
// (DevParams::wall_lo / wall_hi) and is periodic in the index arithmetic
// otherwise; the fused kernel updates only the slab's planes
// (DevParams::zb, ze) and, staging phi one plane beyond them, pulls from the
// ghost planes but never across the local ends.  Which populations cross a
// face is the caller's plan (the host module that drives the exchange):
// the library only copies whole planes in and out.
#include <string.h>

#include "lbmp_internal.h"

namespace {

constexpr int kMaxPlanes = 64;

struct PlaneList {
    long long off[kMaxPlanes];  // element offset of each plane within its population set
    unsigned char set[kMaxPlanes];  // 0: f', 1: g
};

// blockIdx.y = plane k of the list; Pack: sets -> buf, else buf -> sets
template <bool Pack>
__global__ void planes_kernel(float* __restrict__ f, float* __restrict__ g, PlaneList L, int nxy,
                              float* __restrict__ buf)
{
    const int k = blockIdx.y;
    float* base = (L.set[k] ? g : f) + L.off[k];
    float* b = buf + (long long)k * nxy;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nxy; i += gridDim.x * blockDim.x) {
        if (Pack)
            b[i] = base[i];
        else
            base[i] = b[i];
    }
}

int slab_fail(int code, const char* msg) { return lbmp::set_error(code, msg); }

int copy_planes(lbmp_handle* h, const int* plan, int n, float* buf, bool pack)
{
    if (!h) return slab_fail(LBMP_ERR_INVALID_ARG, "null handle");
    if (!plan || !buf) return slab_fail(LBMP_ERR_INVALID_ARG, "null plan or buffer");
    if (n < 0 || n > kMaxPlanes) return slab_fail(LBMP_ERR_INVALID_ARG, "a plan holds 0 to 64 planes");
    if (h->D != 3 || h->params.storage != LBMP_FP32)
        return slab_fail(LBMP_ERR_UNSUPPORTED, "plane copies need a D3Q27 FP32 domain");
    if (n == 0) return LBMP_OK;
    const long long nxy = (long long)h->grid.nx * h->grid.ny;
    PlaneList L;
    memset(&L, 0, sizeof L);
    for (int k = 0; k < n; ++k) {
        const int set = plan[3 * k], a = plan[3 * k + 1], z = plan[3 * k + 2];
        if (set != 0 && set != 1) return slab_fail(LBMP_ERR_INVALID_ARG, "plan: set must be 0 (f') or 1 (g)");
        if (a < 0 || a >= (set ? h->Qg : h->Q)) return slab_fail(LBMP_ERR_INVALID_ARG, "plan: direction out of range");
        if (z < 0 || z >= h->grid.nz) return slab_fail(LBMP_ERR_INVALID_ARG, "plan: plane out of range");
        L.set[k] = (unsigned char)set;
        L.off[k] = (long long)a * h->N + (long long)z * nxy;
    }
    float* f = h->f[h->parity];
    float* g = h->g[h->parity];
    const dim3 grid((unsigned)((nxy + 255) / 256 < 64 ? (nxy + 255) / 256 : 64), (unsigned)n);
    if (pack)
        planes_kernel<true><<<grid, 256, 0, h->stream>>>(f, g, L, (int)nxy, buf);
    else
        planes_kernel<false><<<grid, 256, 0, h->stream>>>(f, g, L, (int)nxy, buf);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return slab_fail(LBMP_ERR_CUDA, cudaGetErrorString(e));
    return LBMP_OK;
}

}  // namespace

extern "C" {

LBMP_API int lbmp_create_slab(const lbmp_grid* grid, int z_begin, int z_end, lbmp_lattice lattice,
                              const lbmp_params* params, void* cuda_stream, const lbmp_allocator* allocator,
                              lbmp_handle** out)
{
    if (!grid || !params || !out) return slab_fail(LBMP_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (lattice != LBMP_D3Q27) return slab_fail(LBMP_ERR_UNSUPPORTED, "z-slabs are D3Q27 domains");
    if (params->storage != LBMP_FP32 || (params->flags & (LBMP_FLAG_PHASE_REDUCED | LBMP_FLAG_DIVU | LBMP_FLAG_AA)))
        return slab_fail(LBMP_ERR_UNSUPPORTED, "z-slabs need FP32 storage, the full phase lattice and no LBMP_FLAG_DIVU");
    if (!(0 <= z_begin && z_begin < z_end && z_end <= grid->nz))
        return slab_fail(LBMP_ERR_INVALID_ARG, "slab planes must satisfy 0 <= z_begin < z_end <= nz");
    if (z_end - z_begin < 2) return slab_fail(LBMP_ERR_INVALID_ARG, "a slab holds at least two planes");
    const bool per = grid->periodic[2] != 0;
    const int glo = (z_begin == 0 && !per) ? 0 : 2;
    const int ghi = (z_end == grid->nz && !per) ? 0 : 2;
    if ((glo == 0 && ghi == 0) || (per && z_begin == 0 && z_end == grid->nz))
        return slab_fail(LBMP_ERR_INVALID_ARG, "a slab borders at least one other slab (else use lbmp_create)");
    lbmp_grid local = *grid;
    local.nz = (z_end - z_begin) + glo + ghi;
    local.periodic[2] = 1;  // index arithmetic only: no updated plane pulls across the local ends
    lbmp_handle* h = nullptr;
    const int rc = lbmp_create_ex(&local, lattice, params, cuda_stream, allocator, &h);
    if (rc != LBMP_OK) return rc;
    lbmp::DevParams& q = h->dp;
    q.wall_lo = glo == 0 ? 1 : 0;
    q.wall_hi = ghi == 0 ? 1 : 0;
    q.zb = glo;
    q.ze = glo + (z_end - z_begin);
    q.zoff = z_begin - glo;
    q.nzg = grid->nz;
    h->slab = true;
    h->slab_z0 = z_begin;
    h->slab_z1 = z_end;
    h->slab_ghost[0] = glo;
    h->slab_ghost[1] = ghi;
    *out = h;
    return LBMP_OK;
}

LBMP_API int lbmp_slab_layout(const lbmp_handle* h, int* layout)
{
    if (!h || !layout) return slab_fail(LBMP_ERR_INVALID_ARG, "null argument");
    const int nv = h->D == 3 ? h->grid.nz : h->grid.ny;
    if (h->slab) {
        layout[0] = h->slab_z0;
        layout[1] = h->slab_z1;
        layout[2] = h->slab_ghost[0];
        layout[3] = h->slab_ghost[1];
    } else {
        layout[0] = 0;
        layout[1] = nv;
        layout[2] = layout[3] = 0;
    }
    layout[4] = nv;
    return LBMP_OK;
}

LBMP_API int lbmp_pack_planes(lbmp_handle* h, const int* plan, int n, float* dev_buf)
{
    return copy_planes(h, plan, n, dev_buf, true);
}

LBMP_API int lbmp_unpack_planes(lbmp_handle* h, const int* plan, int n, const float* dev_buf)
{
    return copy_planes(h, plan, n, const_cast<float*>(dev_buf), false);
}

}  // extern "C"
