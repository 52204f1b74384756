// kern_r_f64.cu -- binary64 local QR without the Gram dot products: the
// R-only form (no Householder vectors or T factors kept; Step 1 of tsqr_r /
// tsqr_svd_values / indirect TSQR on FP64 data and their tree levels) and
// the form that writes Y and tau for the tensor-core Gram (TSQR_PREC_OZAKI).
#define TSQR_S double
#define TSQR_T double
#include "tiles_f64.h"
#define TSQR_LOCAL_R_NAME launch_local_r_f64
#define TSQR_LOCAL_QR_NOGRAM_NAME launch_local_qr_nogram_f64
#include "kern_inst.cuh"
