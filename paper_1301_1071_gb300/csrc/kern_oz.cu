// kern_oz.cu -- launchers of the Ozaki-split tensor-core kernels (binary64
// data): Step 3 and the Gram entries of the T factors.
#define TSQR_OZ_KERNELS
#include "launch.h"
#include "oz_kernels.cuh"

namespace tsqr {

cudaError_t launch_form_q_oz(double* Y, int64_t m, int n, int64_t b, int B, int64_t bt, int kt, int64_t p,
                             const double* T, const double* C, int64_t cblocks, int32_t* status, cudaStream_t st) {
  if (n < 1 || n > kOzMaxN) return cudaErrorInvalidValue;
  const size_t smem = FormQOzSmem(n).total;
  auto fn = oz_k(n) == 16 ? k_form_q_oz<16> : k_form_q_oz<32>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  fn<<<static_cast<unsigned>(p), kOzThreads, smem, st>>>(Y, m, n, static_cast<int>(b), B, static_cast<int>(bt), kt,
                                                         T, C, cblocks, status);
  return cudaGetLastError();
}

cudaError_t launch_gram_oz(const double* Y, int64_t m, int n, int64_t b, int B, int64_t bt, int kt, int64_t p,
                           double* T, int32_t* status, cudaStream_t st) {
  if (n < 1 || n > kGmMaxN) return cudaErrorInvalidValue;
  const size_t smem = GramOzSmem(n).total;
  cudaError_t e = cudaFuncSetAttribute(k_gram_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k_gram_oz<<<static_cast<unsigned>(p), kGmThreads, smem, st>>>(Y, m, n, static_cast<int>(b), B,
                                                                static_cast<int>(bt), kt, T, status);
  return cudaGetLastError();
}

}  // namespace tsqr
