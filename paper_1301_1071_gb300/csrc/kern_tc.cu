// kern_tc.cu -- launcher of the tensor-core Step 3 (binary32 data, 3xTF32):
// k_form_q_tc for n <= 64, the wide form k_form_q_tcw above.
#define TSQR_TC_KERNELS
#include "launch.h"
#include "tc_kernels.cuh"

namespace tsqr {

cudaError_t launch_form_q_tc(float* Y, int64_t m, int n, int64_t b, int B, int64_t bt, int kt, int64_t p,
                             const double* T, const double* C, int64_t cblocks, int32_t* status, cudaStream_t st) {
  if (n < 1 || n > kTcwMaxN) return cudaErrorInvalidValue;
  if (n <= kTcMaxN) {
    const size_t smem = FormQTcSmem(n).total;
    cudaError_t e = cudaFuncSetAttribute(k_form_q_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_form_q_tc<<<static_cast<unsigned>(p), kTcThreads, smem, st>>>(Y, m, n, static_cast<int>(b), B,
                                                                      static_cast<int>(bt), kt, T, C, cblocks, status);
    return cudaGetLastError();
  }
  const size_t smem = FormQTcwSmem(n).total;
  cudaError_t e = cudaFuncSetAttribute(k_form_q_tcw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_form_q_tcw<<<static_cast<unsigned>(p), kTcThreads, smem, st>>>(Y, m, n, static_cast<int>(b), B,
                                                                     static_cast<int>(bt), kt, T, C, cblocks, status);
  return cudaGetLastError();
}

}  // namespace tsqr
