// kern_f32.cu -- binary32 instantiations (Step 1 and Step 3 on FP32 data).
#define TSQR_S float
#define TSQR_T float
#define TSQR_R0 32
#define TSQR_T0 256
#define TSQR_R1 20
#define TSQR_T1 384
#define TSQR_R2 12
#define TSQR_T2 512
#define TSQR_R3 8
#define TSQR_T3 640
#define TSQR_R4 16
#define TSQR_T4 640
#define TSQR_R5 24  // the wide tile: 8 columns per thread (50 < n <= 64)
#define TSQR_T5 256
#define TSQR_N5 8
#define TSQR_R6 10  // 10 columns per thread (n > 64)
#define TSQR_T6 384
#define TSQR_N6 10
#define TSQR_LOCAL_QR_NAME launch_local_qr_f32
#define TSQR_FORM_Q_NAME launch_form_q_f32
#define TSQR_ROWMUL_NAME launch_rowmul_f32
#define TSQR_GRAM_NAME launch_gram_f32
#include "kern_inst.cuh"
