// lbmp_fused_t8x16.cu -- the fused D3Q27 FP32 step and its batch form at a
// 8 x 16 tile (a launch shape of the autotuners; kernel source
// lbmp_fused3_body.cuh).
// Four CTAs (16 warps) per SM at 128 registers: the phase-field outputs
// first, the moment differences parked in the consumed g column, ring phi
// from register loads, pair loops kept in order (measured on the
// 128x128x512 RT workload: 0.852 ms per step against 0.894 ms for three
// CTAs per SM with a separate moment-difference array); column and plane
// offsets in bytes (0.827 against 0.860 ms with element indices)
#define LBMP_FUSED_MINB 4
#define LBMP_FUSED_BYTEOFF 4
#define LBMP_FUSED_SPLIT 1
#define LBMP_FUSED_RINGREG 1
#define LBMP_OUT_ORDERED 1
#define LBMP_FUSED_TX 8
#define LBMP_FUSED_TY 16
#define LBMP_TILE_NS tile8x16
#define LBMP_FUSED3_LAUNCH launch_step_fused3_t8x16
#define LBMP_BATCH3_OPS batch3_ops_8x16
#define LBMP_FUSED3_WITH_COMMON 0
#include "lbmp_fused3_body.cuh"
