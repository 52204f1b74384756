// static_ws.cu -- tsqr_direct_static: direct TSQR whose workspace is a fixed
// array in device memory that the library owns, for callers that cannot
// allocate device memory themselves (a host framework that owns every byte of
// device memory and forbids other allocations, a latency-critical caller that
// cannot afford the implicit device synchronisation of cudaMalloc/cudaFree,
// or plain C code without a device allocator).  This entry point calls no
// allocating routine.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/tsqr.h"

namespace {

constexpr size_t kStaticWorkBytes = static_cast<size_t>(TSQR_STATIC_WORK_BYTES);

// The scratch itself.  Every GPU that loads the library holds these bytes
// until the process exits.  In host code this name is only a stand-in for the
// symbol: its device address is obtained with cudaGetSymbolAddress below.
__device__ __align__(256) unsigned char g_static_work[kStaticWorkBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_static_work on the current device (resolved once per
// device, with that device current).  Returns nullptr on failure.
void* static_work_address(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_work) != cudaSuccess) return nullptr;
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

}  // namespace

extern "C" tsqr_status tsqr_direct_static(const void* A, int64_t m, int64_t n, int64_t lda, int32_t dtype, void* Q,
                                          int64_t ldq, double* R, int64_t ldr, const tsqr_opts* opts,
                                          void* stream) {
  size_t need = 0;
  tsqr_status s = tsqr_workspace_size(TSQR_OP_DIRECT, m, n, dtype, opts, &need);
  if (s != TSQR_OK) return s;
  if (need > kStaticWorkBytes) return TSQR_ERR_WORKSPACE;  // problem too large for the fixed scratch
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
  void* work = static_work_address(dev);
  if (!work) return TSQR_ERR_CUDA;
  // tsqr_direct clears the status word at the start of every call; nothing
  // else in the workspace needs to start at zero.
  return tsqr_direct(A, m, n, lda, dtype, Q, ldq, R, ldr, work, kStaticWorkBytes, opts, stream);
}
