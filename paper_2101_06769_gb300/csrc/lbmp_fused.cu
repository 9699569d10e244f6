// lbmp_fused.cu -- the fused D3Q27 FP32 step and its batch form at the
// default 32 x 4 tile, with the pieces shared by every tile shape (the
// kernel source is lbmp_fused3_body.cuh).
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
#define LBMP_FUSED3_LAUNCH launch_step_fused3
#define LBMP_BATCH3_OPS batch3_ops_32x4
#define LBMP_FUSED3_WITH_COMMON 1
#include "lbmp_fused3_body.cuh"
