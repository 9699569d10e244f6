// lbmp_fused.cu -- the fused D3Q27 FP32 step and its batch form at the
// default 32 x 4 tile, with the pieces shared by every tile shape (the
// kernel source is lbmp_fused3_body.cuh).
#define LBMP_FUSED3_LAUNCH launch_step_fused3
#define LBMP_BATCH3_OPS batch3_ops_32x4
#define LBMP_FUSED3_WITH_COMMON 1
#include "lbmp_fused3_body.cuh"
