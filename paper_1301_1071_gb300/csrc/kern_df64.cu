// kern_df64.cu -- binary64 storage with double-float compute (Step 1 and
// Step 3 on FP64 data in the df64 precision mode; the Gram and row-product
// kernels of the other operations use the binary64 instantiations).
#define TSQR_S double
#define TSQR_T df64
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
#define TSQR_LOCAL_QR_NAME launch_local_qr_df64
#define TSQR_FORM_Q_NAME launch_form_q_df64
#include "kern_inst.cuh"
