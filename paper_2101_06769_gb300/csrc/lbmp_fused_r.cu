// lbmp_fused_r.cu -- the fused D3Q27 FP32 step with the phase field on the
// reduced lattice D3Q7 (first-order equilibrium and correction term,
// Sec. 2.2), 32 x 4 tiles (kernel source lbmp_fused3_body.cuh).  With 7
// instead of 27 staged phase-field values per cell the kernel fits 128
// registers without parking the moment differences in shared memory, so it
// runs four CTAs (16 warps) per SM.
#define LBMP_PHASE_REDUCED 1
#define LBMP_FUSED_MINB 4
#define LBMP_FUSED_DHSMEM 0
#define LBMP_TILE_NS tile_red
#define LBMP_FUSED3_LAUNCH launch_step_fused3_red
#define LBMP_BATCH3_OPS batch3_ops_red
#define LBMP_FUSED3_WITH_COMMON 0
#include "lbmp_fused3_body.cuh"
