// kern_tc.cu -- launcher of the tensor-core Step 3 (binary32 data, 3xTF32):
// k_form_q_tc for n <= 64, the wide form k_form_q_tcw above.
#define TSQR_TC_KERNELS
#include <algorithm>

#include "launch.h"
#include "tc_kernels.cuh"

namespace tsqr {

cudaError_t launch_form_q_tc(float* Y, int64_t m, int n, int64_t b, int B, int64_t bt, int kt, int64_t p,
                             double* T, double* C, int64_t cblocks, int32_t* status, cudaStream_t st) {
  if (n < 1 || n > kTcwMaxN) return cudaErrorInvalidValue;
  if (n <= kTcMaxN) {
    if (cblocks != p) return cudaErrorInvalidValue;  // X_0 goes to each block's own C
    // the W chain (over the T slots and C), then the chunk stream
    const size_t ws = WChainSmem(n).total;
    cudaError_t e = cudaFuncSetAttribute(k_w_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws);
    if (e != cudaSuccess) return e;
    k_w_chain<<<static_cast<unsigned>(p), kWcThreads, ws, st>>>(Y, m, n, b, B, static_cast<int>(bt), kt, T, C,
                                                                 cblocks);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t smem = std::max(FormQTcSmem(n).total, static_cast<size_t>(kTqMinSmem));
    // rows are read and written with the widest vector Y's alignment allows
    const uintptr_t ya = reinterpret_cast<uintptr_t>(Y);
    const int vw = (n % 4 == 0 && (ya & 15) == 0) ? 4 : ((n % 2 == 0 && (ya & 7) == 0) ? 2 : 1);
    // n % 8 == 0: rows at stride n would start on the same banks; they are
    // staged in 16-row groups 16 bytes apart instead (rows 16-byte aligned)
    auto kern = vw == 4 ? (n % 8 == 0 ? k_form_q_tc<4, true> : k_form_q_tc<4, false>)
                        : (vw == 2 ? k_form_q_tc<2, false> : k_form_q_tc<1, false>);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int64_t chunks = TqGeom(m, n, b, B, static_cast<int>(bt), p).total();
    const unsigned grid = static_cast<unsigned>(chunks < sms ? chunks : sms);
    kern<<<grid, kTqThreads, smem, st>>>(Y, m, n, b, B, static_cast<int>(bt), kt, p, T, C, status);
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
