// tiles_f64.h -- the register tiles of the 8-byte kernels (binary64 and
// double-float compute): tile i holds TSQR_Ri rows x TSQR_Ni columns per
// thread (5 unless given) with at most TSQR_Ti threads per CTA.  The
// planner's table (plan.cu, kTiles64) must match.
#pragma once
#define TSQR_R0 16
#define TSQR_T0 256
#define TSQR_R1 10
#define TSQR_T1 384
#define TSQR_R2 6
#define TSQR_T2 512
#define TSQR_R3 4
#define TSQR_T3 640
#define TSQR_R4 8
#define TSQR_T4 640
#define TSQR_R5 12  // the wide tile: 8 columns per thread (50 < n <= 64)
#define TSQR_T5 256
#define TSQR_N5 8
#define TSQR_R6 5  // 10 columns per thread (n > 64)
#define TSQR_T6 384
#define TSQR_N6 10
