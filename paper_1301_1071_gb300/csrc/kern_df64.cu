// kern_df64.cu -- binary64 storage with double-float compute (Step 1 and
// Step 3 on FP64 data in the df64 precision mode).
#define TSQR_S double
#define TSQR_T df64
#define TSQR_R0 12
#define TSQR_T0 320
#define TSQR_R1 8
#define TSQR_T1 448
#define TSQR_R2 4
#define TSQR_T2 640
#define TSQR_R3 8
#define TSQR_T3 640
#define TSQR_LOCAL_QR_NAME launch_local_qr_df64
#define TSQR_FORM_Q_NAME launch_form_q_df64
#define TSQR_ROWMUL_NAME launch_rowmul_df64
#define TSQR_GRAM_NAME launch_gram_df64
#include "kern_inst.cuh"
