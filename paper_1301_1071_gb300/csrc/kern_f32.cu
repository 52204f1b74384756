// kern_f32.cu -- binary32 instantiations (Step 1 and Step 3 on FP32 data).
#define TSQR_S float
#define TSQR_T float
#include "tiles_f32.h"
#define TSQR_LOCAL_QR_NAME launch_local_qr_f32
#define TSQR_FORM_Q_NAME launch_form_q_f32
#define TSQR_ROWMUL_NAME launch_rowmul_f32
#define TSQR_GRAM_NAME launch_gram_f32
#include "kern_inst.cuh"
