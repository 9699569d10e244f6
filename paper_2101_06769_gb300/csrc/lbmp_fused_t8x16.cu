// lbmp_fused_t8x16.cu -- the fused D3Q27 FP32 step and its batch form at a
// 8 x 16 tile (a launch shape of the autotuners; kernel source
// lbmp_fused3_body.cuh).
#define LBMP_FUSED_TX 8
#define LBMP_FUSED_TY 16
#define LBMP_TILE_NS tile8x16
#define LBMP_FUSED3_LAUNCH launch_step_fused3_t8x16
#define LBMP_BATCH3_OPS batch3_ops_8x16
#define LBMP_FUSED3_WITH_COMMON 0
#include "lbmp_fused3_body.cuh"
