// kern_r_f32.cu -- binary32 R-only local QR (no Householder vectors or T
// factors kept): Step 1 of tsqr_r / tsqr_svd_values / indirect TSQR on FP32
// data.
#define TSQR_S float
#define TSQR_T float
#include "tiles_f32.h"
#define TSQR_LOCAL_R_NAME launch_local_r_f32
#include "kern_inst.cuh"
