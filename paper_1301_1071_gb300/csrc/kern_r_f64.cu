// kern_r_f64.cu -- binary64 R-only local QR (no Householder vectors or T
// factors kept): Step 1 of tsqr_r / tsqr_svd_values / indirect TSQR on FP64
// data and their tree levels.
#define TSQR_S double
#define TSQR_T double
#include "tiles_f64.h"
#define TSQR_LOCAL_R_NAME launch_local_r_f64
#include "kern_inst.cuh"
