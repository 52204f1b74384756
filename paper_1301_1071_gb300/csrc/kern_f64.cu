// kern_f64.cu -- binary64 instantiations (Step 1 on FP64 data and every
// Step-2 tree level).
#define TSQR_S double
#define TSQR_T double
#include "tiles_f64.h"
#define TSQR_LOCAL_QR_NAME launch_local_qr_f64
#define TSQR_FORM_Q_NAME launch_form_q_f64
#define TSQR_ROWMUL_NAME launch_rowmul_f64
#define TSQR_GRAM_NAME launch_gram_f64
#include "kern_inst.cuh"
