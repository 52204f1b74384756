// kern_df64.cu -- binary64 storage with double-float compute (Step 1 and
// Step 3 on FP64 data in the df64 precision mode; the Gram and row-product
// kernels of the other operations use the binary64 instantiations).
#define TSQR_S double
#define TSQR_T df64
#include "tiles_f64.h"
#define TSQR_LOCAL_QR_NAME launch_local_qr_df64
#define TSQR_FORM_Q_NAME launch_form_q_df64
#include "kern_inst.cuh"
