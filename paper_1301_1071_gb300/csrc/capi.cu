// capi.cu -- the extern "C" boundary (include/tsqr.h): argument checks, the
// plan, and the launch sequence of each computation on the caller's stream.
#include <atomic>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <cuda_runtime.h>

#include "../../include/tsqr.h"
#include "check.h"
#include "launch.h"
#include "plan.h"
#include "small.cuh"
#include "tc_kernels.cuh"

namespace tsqr {

cudaError_t launch_local_qr_f64(const KernelCfg&, const void*, int64_t, int, int64_t, int64_t, int, int64_t, void*, double*,
                                double*, int32_t*, cudaStream_t);
cudaError_t launch_local_qr_f32(const KernelCfg&, const void*, int64_t, int, int64_t, int64_t, int, int64_t, void*, double*,
                                double*, int32_t*, cudaStream_t);
cudaError_t launch_form_q_f64(const KernelCfg&, const void*, int64_t, int, int64_t, int64_t, int, int64_t, const double*,
                              const double*, int64_t, void*, int32_t*, cudaStream_t);
cudaError_t launch_form_q_f32(const KernelCfg&, const void*, int64_t, int, int64_t, int64_t, int, int64_t, const double*,
                              const double*, int64_t, void*, int32_t*, cudaStream_t);

cudaError_t launch_local_qr_df64(const KernelCfg&, const void*, int64_t, int, int64_t, int64_t, int, int64_t, void*, double*,
                                 double*, int32_t*, cudaStream_t);
cudaError_t launch_form_q_df64(const KernelCfg&, const void*, int64_t, int, int64_t, int64_t, int, int64_t, const double*,
                               const double*, int64_t, void*, int32_t*, cudaStream_t);
cudaError_t launch_local_r_f64(const KernelCfg&, const void*, int64_t, int, int64_t, int64_t, int, int64_t, double*,
                               int32_t*, cudaStream_t);
cudaError_t launch_local_r_f32(const KernelCfg&, const void*, int64_t, int, int64_t, int64_t, int, int64_t, double*,
                               int32_t*, cudaStream_t);
cudaError_t launch_local_qr_nogram_f64(const KernelCfg&, const void*, int64_t, int, int64_t, int64_t, int, int64_t,
                                       void*, double*, double*, int32_t*, cudaStream_t);
cudaError_t launch_rowmul_f64(const KernelCfg&, const void*, const double*, const void*, const double*, int64_t,
                              int, int64_t, int64_t, void*, int32_t*, cudaStream_t);
cudaError_t launch_rowmul_f32(const KernelCfg&, const void*, const double*, const void*, const double*, int64_t,
                              int, int64_t, int64_t, void*, int32_t*, cudaStream_t);
cudaError_t launch_gram_f64(const void*, const void*, int64_t, int, int, int, int, int, bool, double*, int32_t*,
                            cudaStream_t);
cudaError_t launch_gram_f32(const void*, const void*, int64_t, int, int, int, int, int, bool, double*, int32_t*,
                            cudaStream_t);

cudaError_t launch_rowmul(const KernelCfg& k, const void* X, const double* M1, const void* Y,
                          const double* M2, int64_t m, int n, int64_t b, int64_t p, void* out, int32_t* status,
                          cudaStream_t st) {
  return k.kind == kKindF32 ? launch_rowmul_f32(k, X, M1, Y, M2, m, n, b, p, out, status, st)
                            : launch_rowmul_f64(k, X, M1, Y, M2, m, n, b, p, out, status, st);
}

cudaError_t launch_gram(int esz, const void* X, const void* Y, int64_t m, int n, double* part, double* G,
                        int32_t* status, cudaStream_t st, bool acc_storage) {
  const GramGeom g = gram_geom(m, n, esz);
  cudaError_t e =
      esz == 8 ? launch_gram_f64(X, Y, m, n, g.chunk, g.grid, g.nt, g.tile, acc_storage, part, status, st)
               : launch_gram_f32(X, Y, m, n, g.chunk, g.grid, g.nt, g.tile, acc_storage, part, status, st);
  if (e != cudaSuccess) return e;
  return launch_gram_reduce(part, g.grid, n, G, status, st);
}

cudaError_t launch_local_qr(const KernelCfg& k, const void* A, int64_t m, int n, int64_t b, int64_t bt, int kt,
                            int64_t p, void* Y, double* Rst, double* Tst, int32_t* status, cudaStream_t st) {
  // R only (Y == NULL) on a one-row-group tile: the form without Gram dot products
  const bool r_only = Y == nullptr && k.NRG == 1;
  switch (k.kind) {
    case kKindF64:
      return r_only ? launch_local_r_f64(k, A, m, n, b, bt, kt, p, Rst, status, st)
                    : launch_local_qr_f64(k, A, m, n, b, bt, kt, p, Y, Rst, Tst, status, st);
    case kKindF32:
      return r_only ? launch_local_r_f32(k, A, m, n, b, bt, kt, p, Rst, status, st)
                    : launch_local_qr_f32(k, A, m, n, b, bt, kt, p, Y, Rst, Tst, status, st);
    case kKindDF64: return launch_local_qr_df64(k, A, m, n, b, bt, kt, p, Y, Rst, Tst, status, st);
    default: return cudaErrorInvalidValue;
  }
}

// Step 1 of direct TSQR: Y_i, R_i and the T slots' tau and Gram entries (the
// Ozaki form: the Gram entries on the tensor cores after a Step 1 without
// them).
// The Householder kernel of Step 1 alone (without its Gram dot products in
// the Ozaki form).
cudaError_t launch_local_qr_step1(const Plan& P, const void* A, int64_t m, int64_t b, int64_t p, void* Y,
                                  double* Rst, double* Tst, int32_t* status, cudaStream_t st) {
  const Level& l0 = P.levels[0];
  const int n = static_cast<int>(P.n);
  if (!P.gram_oz) return launch_local_qr(P.cfg0, A, m, n, b, l0.bt, l0.kt, p, Y, Rst, Tst, status, st);
  return launch_local_qr_nogram_f64(P.cfg0, A, m, n, b, l0.bt, l0.kt, p, Y, Rst, Tst, status, st);
}

cudaError_t launch_step1(const Plan& P, const void* A, int64_t m, int64_t b, int64_t p, void* Y, double* Rst,
                         double* Tst, int32_t* status, cudaStream_t st) {
  const Level& l0 = P.levels[0];
  const int n = static_cast<int>(P.n);
  cudaError_t e = launch_local_qr_step1(P, A, m, b, p, Y, Rst, Tst, status, st);
  if (e != cudaSuccess || !P.gram_oz) return e;
  return launch_gram_oz(static_cast<const double*>(Y), m, n, b, P.cfg0.B, l0.bt, l0.kt, p, Tst, status, st);
}

cudaError_t launch_form_q(const KernelCfg& k, const void* Y, int64_t m, int n, int64_t b, int64_t bt, int kt,
                          int64_t p, const double* T, const double* C, int64_t cblocks, void* Q, int32_t* status,
                          cudaStream_t st) {
  switch (k.kind) {
    case kKindF64: return launch_form_q_f64(k, Y, m, n, b, bt, kt, p, T, C, cblocks, Q, status, st);
    case kKindF32: return launch_form_q_f32(k, Y, m, n, b, bt, kt, p, T, C, cblocks, Q, status, st);
    case kKindDF64: return launch_form_q_df64(k, Y, m, n, b, bt, kt, p, T, C, cblocks, Q, status, st);
    default: return cudaErrorInvalidValue;
  }
}

namespace {

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
// NULL (an optional argument left out) or 16-byte aligned
bool aligned16_or_null(const void* p) { return p == nullptr || aligned16(p); }

// SM count of the current device (the planner's default block height
// depends on it); the GB300 value when no device answers.
int device_sms() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return kDefaultSMs;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
    cudaGetLastError();  // clear the error of a host without a device
    return kDefaultSMs;
  }
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

int esz_of(int32_t dtype) { return dtype == TSQR_F64 ? 8 : (dtype == TSQR_F32 ? 4 : 0); }

tsqr_status check_opts(const tsqr_opts* o) {
  if (!o) return TSQR_OK;
  if (o->reserved != 0) return TSQR_ERR_ARG;
  if (o->prec < TSQR_PREC_NATIVE || o->prec > TSQR_PREC_OZAKI) return TSQR_ERR_ARG;
  if (o->block_rows < 0 || o->tree_fanout < 0 || o->tree_fanout == 1) return TSQR_ERR_ARG;
  return TSQR_OK;
}

// Ops whose plan follows opts->prec (the others compute in the data's type).
bool op_takes_prec(int op) {
  return op == TSQR_OP_DIRECT || op == TSQR_OP_SVD || op == TSQR_OP_DIRECT_HOST || op == TSQR_OP_R ||
         op == TSQR_OP_SVD_VALUES;
}

char* at(void* work, size_t off) { return static_cast<char*>(work) + off; }

int32_t* status_ptr(void* work) { return reinterpret_cast<int32_t*>(work); }

tsqr_status finish(void* work, const tsqr_opts* o, cudaStream_t st) {
  if (cudaGetLastError() != cudaSuccess) return TSQR_ERR_CUDA;
  if (o && o->sync) return tsqr_read_status(work, st);
  return TSQR_OK;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = static_cast<const char*>(a);
  const char* pb = static_cast<const char*>(b);
  return pa < pb + nb && pb < pa + na;
}

// An m x n matrix whose byte size at 8 bytes an entry int64 holds (the
// planner, the overlap checks and the kernels index with it).
bool rows_fit(int64_t m, int64_t n) { return n >= 1 && m <= INT64_MAX / 8 / n; }

// Shared argument checks of the tall-matrix entry points.
tsqr_status check_tall(const void* A, int64_t m, int64_t n, int64_t lda, int32_t dtype, const tsqr_opts* o) {
  if (!A) return TSQR_ERR_ARG;
  if (esz_of(dtype) == 0) return TSQR_ERR_ARG;
  tsqr_status s = check_opts(o);
  if (s != TSQR_OK) return s;
  if (n < 1 || n > TSQR_NMAX || m < n || !rows_fit(m, n)) return TSQR_ERR_SHAPE;
  if (lda != n || !aligned16(A)) return TSQR_ERR_ALIGN;
  return TSQR_OK;
}

// Direct TSQR on a built plan.  extra(ctop, stream) is launched on the tree's
// stream between the sign fix and the down pass (the SVD variant folds U_R
// into Ctop there).
tsqr_status mark(const tsqr_opts* o, int i, cudaStream_t st) {
  if (!o || !o->stage_events || !o->stage_events[i]) return TSQR_OK;
  return cudaEventRecord(static_cast<cudaEvent_t>(o->stage_events[i]), st) == cudaSuccess ? TSQR_OK
                                                                                          : TSQR_ERR_CUDA;
}

#define TSQR_TRY(x)                       \
  do {                                    \
    tsqr_status _s = (x);                 \
    if (_s != TSQR_OK) return _s;         \
  } while (0)
#define TSQR_CUDA(x) TSQR_TRY((x) == cudaSuccess ? TSQR_OK : TSQR_ERR_CUDA)

// A second stream (the device's highest priority) for the Step-2 tree: one
// per device, created on first use and kept until the process exits, and a
// fork / join event pair per call.  Once forked, the guard's destructor
// always records the join on the side stream and makes the caller's stream
// wait for it, on every exit path (an error after the fork included), so
// that work queued on the side stream is never left unordered with `stream`.
constexpr size_t kOverlapTBytes = static_cast<size_t>(TSQR_STATIC_WORK_BYTES);  // 16 MiB of T slots

cudaStream_t device_side_stream() {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static cudaStream_t streams[kMaxDev] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!streams[dev]) {
    int least = 0, greatest = 0;
    cudaStream_t s = nullptr;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, greatest) != cudaSuccess)
      return nullptr;
    streams[dev] = s;
  }
  return streams[dev];
}

struct SideStream {
  cudaStream_t s = nullptr, caller = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  bool forked = false;
  // Forks the side stream from `st`: false (nothing forked) on failure.
  bool make(cudaStream_t st) {
    caller = st;
    s = device_side_stream();
    if (!s || cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess)
      return false;
    if (cudaEventRecord(fork, st) != cudaSuccess || cudaStreamWaitEvent(s, fork, 0) != cudaSuccess) return false;
    forked = true;
    return true;
  }
  // Orders the caller's stream after everything queued on the side stream.
  cudaError_t rejoin() {
    if (!forked) return cudaSuccess;
    forked = false;
    cudaError_t e = cudaEventRecord(join, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, join, 0);
    // an ordering that cannot be expressed with the event: wait on the host
    if (e != cudaSuccess) cudaStreamSynchronize(s);
    return e;
  }
  ~SideStream() {
    rejoin();
    if (join) cudaEventDestroy(join);  // released by the driver once its work has completed
    if (fork) cudaEventDestroy(fork);
  }
};

// Step 2 (Alg. 2) after Step 1 has filled the level-0 stack: the tree up
// (each level's stack is the tall input of the next), the top sign fix into
// R, `extra` on the top coefficient, and the tree down (the Q of level l's
// stack is the coefficient of level l - 1), leaving Step 3's coefficients.
template <class Extra>
tsqr_status run_tree(const Plan& P, double* R, int64_t ldr, void* work, cudaStream_t st, Extra extra) {
  const int n = static_cast<int>(P.n);
  int32_t* status = status_ptr(work);
  const size_t L = P.levels.size();
  auto S = [&](size_t l) { return reinterpret_cast<double*>(at(work, P.levels[l].off_S)); };
  auto T = [&](size_t l) { return reinterpret_cast<double*>(at(work, P.levels[l].off_T)); };
  double* ctop = reinterpret_cast<double*>(at(work, P.off_ctop));
  for (size_t l = 1; l < L; ++l) {
    const Level& lv = P.levels[l];
    // a node is f stacked triangles: the structured factorisation (tree.cu)
    // in one CTA's shared memory, else over a cluster of f CTAs
    const int f = static_cast<int>(lv.b / n);
    const cudaError_t e =
        tree_up_fits(n, f)      ? launch_tree_up(S(l - 1), lv.rows, n, f, lv.p, S(l - 1), S(l), T(l), st)
        : tree_up_cl_fits(n, f) ? launch_tree_up_cl(S(l - 1), lv.rows, n, f, lv.p, S(l - 1), S(l), T(l), st)
                                : launch_local_qr(P.cfg64, S(l - 1), lv.rows, n, lv.b, lv.bt, lv.kt, lv.p, S(l - 1),
                                                  S(l), T(l), status, st);
    if (e != cudaSuccess) return TSQR_ERR_CUDA;
    if (launch_build_t(T(l), lv.p * lv.kt, n, false, st) != cudaSuccess) return TSQR_ERR_CUDA;
  }
  if (launch_sign_fix(S(L - 1), n, R, ldr, ctop, status, st) != cudaSuccess) return TSQR_ERR_CUDA;
  if (extra(ctop, st) != TSQR_OK) return TSQR_ERR_CUDA;
  for (size_t l = L - 1; l >= 1; --l) {
    const Level& lv = P.levels[l];
    const double* C = (l == L - 1) ? ctop : S(l);
    const int64_t cb = (l == L - 1) ? 1 : lv.p;
    // a node is f stacked triangles: the structured product (tree.cu)
    const cudaError_t e = launch_tree_down(S(l - 1), lv.rows, n, static_cast<int>(lv.b / n), lv.p, T(l), C, cb, st);
    if (e != cudaSuccess) return TSQR_ERR_CUDA;
  }
  return TSQR_OK;
}

template <class Extra>
tsqr_status run_direct(const Plan& P, const void* A, void* Q, double* R, int64_t ldr, void* work,
                       cudaStream_t st, const tsqr_opts* o, Extra extra) {
  const int n = static_cast<int>(P.n);
  int32_t* status = status_ptr(work);
  if (cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) return TSQR_ERR_CUDA;
  const size_t L = P.levels.size();
  auto S = [&](size_t l) { return reinterpret_cast<double*>(at(work, P.levels[l].off_S)); };
  auto T = [&](size_t l) { return reinterpret_cast<double*>(at(work, P.levels[l].off_T)); };
  double* ctop = reinterpret_cast<double*>(at(work, P.off_ctop));

  // Step 1: local QR of every row block; Y_0 is written into Q's storage.
  const Level& l0 = P.levels[0];
  if (mark(o, 0, st) != TSQR_OK) return TSQR_ERR_CUDA;
  if (launch_local_qr_step1(P, A, P.m, l0.b, l0.p, Q, S(0), T(0), status, st) != cudaSuccess) return TSQR_ERR_CUDA;
  if (mark(o, 1, st) != TSQR_OK) return TSQR_ERR_CUDA;
  // the T factors' Gram entries on the tensor cores (Ozaki form); like the T
  // build below, it is part of the Step-2 interval of the stage events
  if (P.gram_oz && launch_gram_oz(static_cast<const double*>(Q), P.m, n, l0.b, P.cfg0.B, l0.bt, l0.kt, l0.p, T(0),
                                  status, st) != cudaSuccess)
    return TSQR_ERR_CUDA;
  // The row blocks' T factors are read only by Step 3 and the tree reads only
  // the stack of R factors, so for a large T build the tree runs on a side
  // stream of the device's highest priority beside it: the block scheduler
  // starts the tree's pending CTAs ahead of the T build's as SMs free up, and
  // the T build fills the SMs the tree's upper levels leave idle.  Step 3
  // waits for both.  Small builds stay in line: they take less time than the
  // side stream's set-up is worth (and no workspace of tsqr_direct_static, at
  // most TSQR_STATIC_WORK_BYTES, reaches the threshold).
  const bool overlap_t = static_cast<size_t>(l0.p) * l0.kt * n * n * sizeof(double) >= kOverlapTBytes;
  SideStream side;  // on every exit after a fork, `st` is made to wait for the side stream
  cudaStream_t tree_st = st;
  if (overlap_t) {
    if (!side.make(st)) return TSQR_ERR_CUDA;
    tree_st = side.s;
  }
  if (launch_build_t(T(0), l0.p * l0.kt, n, P.esz == 4, st) != cudaSuccess) return TSQR_ERR_CUDA;
  TSQR_TRY(run_tree(P, R, ldr, work, tree_st, extra));
  TSQR_CUDA(side.rejoin());
  // Step 3: Q_i = Q1_i Q2_i over the Y_i held in Q.
  if (mark(o, 2, st) != TSQR_OK) return TSQR_ERR_CUDA;
  double* C0 = (L == 1) ? ctop : S(0);
  const int64_t cb0 = (L == 1) ? 1 : l0.p;
  const cudaError_t e3 =
      P.oz3   ? launch_form_q_oz(static_cast<double*>(Q), P.m, n, l0.b, P.cfg0.B, l0.bt, l0.kt, l0.p, T(0), C0, cb0,
                                 status, st)
      : P.tc3 ? launch_form_q_tc(static_cast<float*>(Q), P.m, n, l0.b, P.cfg0.B, l0.bt, l0.kt, l0.p, T(0), C0, cb0,
                                 status, st)
              : launch_form_q(P.cfg0, Q, P.m, n, l0.b, l0.bt, l0.kt, l0.p, T(0), C0, cb0, Q, status, st);
  if (e3 != cudaSuccess) return TSQR_ERR_CUDA;
  return mark(o, 3, st);
}

// R factor only (indirect TSQR, Sec. II-B): Steps 1-2 without Y/T/Q2, then
// the sign normalisation into R (n x n, leading dimension n).  `ctop` receives
// the (unused) sign matrix.
tsqr_status run_r_only(const Plan& P, int esz, const void* X, double* R, void* work, cudaStream_t st) {
  const int n = static_cast<int>(P.n);
  int32_t* status = status_ptr(work);
  const size_t L = P.levels.size();
  auto S = [&](size_t l) { return reinterpret_cast<double*>(at(work, P.levels[l].off_S)); };
  double* ctop = reinterpret_cast<double*>(at(work, P.off_ctop));
  const Level& l0 = P.levels[0];
  const cudaError_t e0 =
      launch_local_qr(P.cfg0, X, P.m, n, l0.b, l0.bt, l0.kt, l0.p, nullptr, S(0), nullptr, status, st);
  if (e0 != cudaSuccess) return TSQR_ERR_CUDA;
  for (size_t l = 1; l < L; ++l) {
    const Level& lv = P.levels[l];
    const int f = static_cast<int>(lv.b / n);
    const cudaError_t e =
        tree_up_fits(n, f)      ? launch_tree_up(S(l - 1), lv.rows, n, f, lv.p, nullptr, S(l), nullptr, st)
        : tree_up_cl_fits(n, f) ? launch_tree_up_cl(S(l - 1), lv.rows, n, f, lv.p, nullptr, S(l), nullptr, st)
                                : launch_local_qr(P.cfg64, S(l - 1), lv.rows, n, lv.b, lv.bt, lv.kt, lv.p, nullptr,
                                                  S(l), nullptr, status, st);
    if (e != cudaSuccess) return TSQR_ERR_CUDA;
  }
  if (launch_sign_fix(S(L - 1), n, R, n, ctop, status, st) != cudaSuccess) return TSQR_ERR_CUDA;
  return TSQR_OK;
}

// out = X M1 (+ Y M2): one input over the row blocks of the Step-1
// configuration; two inputs with the tile sized for two staged inputs.
tsqr_status rowmul(const Plan& P, const void* X, const double* M1, const void* Y, const double* M2, void* out,
                   int32_t* status, cudaStream_t st) {
  const bool two = X && Y;
  const KernelCfg& k = two ? P.cfg_rm2 : P.cfg0;
  const int64_t b = two ? P.b_rm2 : P.cfg0.rm_rows;
  const int64_t p = (P.m + b - 1) / b;
  return launch_rowmul(k, X, M1, Y, M2, P.m, (int)P.n, b, p, out, status, st) == cudaSuccess
             ? TSQR_OK
             : TSQR_ERR_CUDA;
}

tsqr_status copy_r(double* R, int64_t ldr, const double* src, int64_t n, cudaStream_t st) {
  return cudaMemcpy2DAsync(R, ldr * sizeof(double), src, n * sizeof(double), n * sizeof(double), n,
                           cudaMemcpyDeviceToDevice, st) == cudaSuccess
             ? TSQR_OK
             : TSQR_ERR_CUDA;
}

// tsqr_direct_host on a built plan: chunk c covers row blocks
// [c pc, (c + 1) pc).  Step 1 and Step 3 of a chunk run as one launch each
// over that chunk's blocks (pointer offsets; the kernels index blocks from 0).
struct HostEvents {
  cudaEvent_t ev[2 * kMaxHostChunks + 1] = {};
  int count = 0;
  ~HostEvents() {
    for (int i = 0; i < count; ++i) cudaEventDestroy(ev[i]);  // released once their work completes
  }
  bool make(int k) {
    for (; count < k; ++count)
      if (cudaEventCreateWithFlags(&ev[count], cudaEventDisableTiming) != cudaSuccess) return false;
    return true;
  }
};

// Once work is queued on the copy stream, every exit (an error included)
// records `ev` on it and makes `st` wait for it (or, if that cannot be
// enqueued, waits for the copy stream on the host), so that the call stays
// ordered on `stream` alone.
struct CopyJoin {
  cudaStream_t cst = nullptr, st = nullptr;
  cudaEvent_t ev = nullptr;
  bool armed = false;
  cudaError_t join() {
    if (!armed) return cudaSuccess;
    armed = false;
    cudaError_t e = cudaEventRecord(ev, cst);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
    if (e != cudaSuccess) cudaStreamSynchronize(cst);
    return e;
  }
  ~CopyJoin() { join(); }
};

tsqr_status run_direct_host(const Plan& P, int chunks, const char* A, char* Qh, double* Rh, char* dbuf, void* work,
                            cudaStream_t st, cudaStream_t cst) {
  const int n = static_cast<int>(P.n);
  const size_t row_bytes = (size_t)n * P.esz;
  const size_t nn = (size_t)n * n;
  int32_t* status = status_ptr(work);
  const Level& l0 = P.levels[0];
  const size_t L = P.levels.size();
  double* S0 = reinterpret_cast<double*>(at(work, l0.off_S));
  double* T0 = reinterpret_cast<double*>(at(work, l0.off_T));
  double* ctop = reinterpret_cast<double*>(at(work, P.off_ctop));
  double* Rd = reinterpret_cast<double*>(at(work, P.off_small));
  const int64_t pc = (l0.p + chunks - 1) / chunks;
  HostEvents E;
  if (!E.make(2 * chunks + 1)) return TSQR_ERR_CUDA;
  cudaEvent_t* ev_in = E.ev;             // chunk's rows of A are on the device
  cudaEvent_t* ev_q = E.ev + chunks;     // chunk's rows of Q are formed
  cudaEvent_t ev_done = E.ev[2 * chunks];
  TSQR_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  // the copy stream must not overwrite dbuf before earlier work on `stream` is done
  TSQR_CUDA(cudaEventRecord(ev_done, st));
  TSQR_CUDA(cudaStreamWaitEvent(cst, ev_done, 0));
  CopyJoin join;  // declared after E: joins before the events are released
  join.cst = cst;
  join.st = st;
  join.ev = ev_done;
  join.armed = true;
  auto chunk_rows = [&](int c, int64_t* b0, int64_t* pcnt, int64_t* r0, int64_t* rows) {
    *b0 = c * pc;
    *pcnt = (l0.p - *b0 < pc) ? l0.p - *b0 : pc;
    *r0 = *b0 * l0.b;
    const int64_t r1 = (*b0 + *pcnt) * l0.b;
    *rows = (r1 < P.m ? r1 : P.m) - *r0;
  };
  // Step 1, chunk by chunk as A's rows arrive
  for (int c = 0; c < chunks; ++c) {
    int64_t b0, pcnt, r0, rows;
    chunk_rows(c, &b0, &pcnt, &r0, &rows);
    if (pcnt <= 0) continue;
    TSQR_CUDA(cudaMemcpyAsync(dbuf + r0 * row_bytes, A + r0 * row_bytes, rows * row_bytes, cudaMemcpyHostToDevice,
                              cst));
    TSQR_CUDA(cudaEventRecord(ev_in[c], cst));
    TSQR_CUDA(cudaStreamWaitEvent(st, ev_in[c], 0));
    TSQR_CUDA(launch_step1(P, dbuf + r0 * row_bytes, rows, l0.b, pcnt, dbuf + r0 * row_bytes, S0 + b0 * nn,
                           T0 + b0 * l0.kt * nn, status, st));
    TSQR_CUDA(launch_build_t(T0 + b0 * l0.kt * nn, pcnt * l0.kt, n, P.esz == 4, st));
  }
  // Step 2, then R back to the host
  TSQR_TRY(run_tree(P, Rd, n, work, st, [](double*, cudaStream_t) { return TSQR_OK; }));
  TSQR_CUDA(cudaMemcpyAsync(Rh, Rd, nn * sizeof(double), cudaMemcpyDeviceToHost, st));
  // Step 3, chunk by chunk, each chunk of Q copied back behind the next
  double* C0 = (L == 1) ? ctop : S0;
  for (int c = 0; c < chunks; ++c) {
    int64_t b0, pcnt, r0, rows;
    chunk_rows(c, &b0, &pcnt, &r0, &rows);
    if (pcnt <= 0) continue;
    double* Cc = (L == 1) ? C0 : C0 + b0 * nn;
    const int64_t cb = (L == 1) ? 1 : pcnt;
    char* Y = dbuf + r0 * row_bytes;
    TSQR_CUDA(P.oz3   ? launch_form_q_oz(reinterpret_cast<double*>(Y), rows, n, l0.b, P.cfg0.B, l0.bt, l0.kt, pcnt,
                                         T0 + b0 * l0.kt * nn, Cc, cb, status, st)
              : P.tc3 ? launch_form_q_tc(reinterpret_cast<float*>(Y), rows, n, l0.b, P.cfg0.B, l0.bt, l0.kt, pcnt,
                                         T0 + b0 * l0.kt * nn, Cc, cb, status, st)
                      : launch_form_q(P.cfg0, Y, rows, n, l0.b, l0.bt, l0.kt, pcnt, T0 + b0 * l0.kt * nn, Cc, cb, Y,
                                      status, st));
    TSQR_CUDA(cudaEventRecord(ev_q[c], st));
    TSQR_CUDA(cudaStreamWaitEvent(cst, ev_q[c], 0));
    TSQR_CUDA(cudaMemcpyAsync(Qh + r0 * row_bytes, Y, rows * row_bytes, cudaMemcpyDeviceToHost, cst));
  }
  TSQR_CUDA(join.join());
  return TSQR_OK;
}

tsqr_status plan_for(int op, int64_t m, int64_t n, int32_t dtype, const tsqr_opts* o, size_t work_bytes,
                     const void* work, Plan* P) {
  const int prec = (o && op_takes_prec(op)) ? o->prec : 0;
  int rc = make_plan(m, n, esz_of(dtype), o ? o->block_rows : 0, o ? o->tree_fanout : 0, P, prec,
                     device_sms());
  if (rc != TSQR_OK) return static_cast<tsqr_status>(rc);
  if (!work || !aligned16(work) || work_bytes < op_bytes(*P, op)) return TSQR_ERR_WORKSPACE;
  return TSQR_OK;
}

}  // namespace
}  // namespace tsqr

using namespace tsqr;

extern "C" {

const char* tsqr_status_string(int32_t s) {
  switch (s) {
    case TSQR_OK: return "TSQR_OK";
    case TSQR_ERR_ARG: return "TSQR_ERR_ARG: invalid argument";
    case TSQR_ERR_SHAPE: return "TSQR_ERR_SHAPE: unsupported shape";
    case TSQR_ERR_ALIGN: return "TSQR_ERR_ALIGN: leading dimension or alignment";
    case TSQR_ERR_WORKSPACE: return "TSQR_ERR_WORKSPACE: workspace missing or too small";
    case TSQR_ERR_CUDA: return "TSQR_ERR_CUDA: CUDA runtime error";
    case TSQR_ERR_NOT_SPD: return "TSQR_ERR_NOT_SPD: Cholesky breakdown";
    case TSQR_ERR_SINGULAR: return "TSQR_ERR_SINGULAR: zero diagonal in R";
    case TSQR_ERR_NONFINITE: return "TSQR_ERR_NONFINITE: NaN or Inf";
    case TSQR_ERR_TIMEOUT: return "TSQR_ERR_TIMEOUT: bounded wait expired";
    case TSQR_ERR_NOCONV: return "TSQR_ERR_NOCONV: Jacobi SVD did not converge";
    default: return "unknown tsqr_status";
  }
}

tsqr_status tsqr_launch_count(int32_t op, int64_t m, int64_t n, int32_t dtype, const tsqr_opts* opts,
                              int32_t refine_steps, int32_t* launches) {
  if (!launches || refine_steps < 0) return TSQR_ERR_ARG;
  const int esz = esz_of(dtype);
  if (esz == 0) return TSQR_ERR_ARG;
  tsqr_status s = check_opts(opts);
  if (s != TSQR_OK) return s;
  if (op == TSQR_OP_ACCURACY) {
    if (n < 1 || n > TSQR_NMAX || m < 1) return TSQR_ERR_SHAPE;
    *launches = 2;  // partial sums, ordered combination
    return TSQR_OK;
  }
  const int prec = (opts && op_takes_prec(op)) ? opts->prec : 0;
  Plan P;
  int chunks = 1;
  int rc = op == TSQR_OP_DIRECT_HOST
               ? make_host_plan(m, n, esz, opts ? opts->block_rows : 0, opts ? opts->tree_fanout : 0, &P, &chunks,
                                prec, device_sms())
               : make_plan(m, n, esz, opts ? opts->block_rows : 0, opts ? opts->tree_fanout : 0, &P, prec,
                           device_sms());
  if (rc != TSQR_OK) return static_cast<tsqr_status>(rc);
  const int L = static_cast<int>(P.levels.size());
  const int g = P.gram_oz ? 1 : 0;                     // the tensor-core Gram after Step 1
  const int w = (P.tc3 && P.n <= kTcMaxN) ? 1 : 0;  // the W chain before the 3xTF32 chunk stream
  switch (op) {
    case TSQR_OP_DIRECT_HOST: *launches = (3 + g + w) * chunks + 3 * (L - 1) + 1; break;  // chunks x (Step 1, T, Step 3)
    case TSQR_OP_DIRECT: *launches = 3 * L + 1 + g + w; break;    // L up (+ T build), sign fix, L down
    case TSQR_OP_SVD: *launches = 3 * L + 2 + g + w; break;       // + Jacobi SVD
    case TSQR_OP_CHOLQR: *launches = 4 * (1 + refine_steps) + refine_steps; break;  // gram, reduce, chol, rowmul (+ combine)
    case TSQR_OP_INDIRECT: *launches = (L + 3) * (1 + refine_steps) + refine_steps; break;
    case TSQR_OP_BACKWARD: *launches = 4; break;              // gram, reduce, prep, rowmul
    case TSQR_OP_R: *launches = L + 1; break;                 // L levels up (R only), sign fix
    case TSQR_OP_SVD_VALUES: *launches = L + 2; break;        // + Jacobi SVD
    default: return TSQR_ERR_ARG;
  }
  return TSQR_OK;
}

tsqr_status tsqr_plan_query(int32_t op, int64_t m, int64_t n, int32_t dtype, const tsqr_opts* opts,
                            tsqr_plan_info* info) {
  if (!info) return TSQR_ERR_ARG;
  const int esz = esz_of(dtype);
  if (esz == 0) return TSQR_ERR_ARG;
  tsqr_status s = check_opts(opts);
  if (s != TSQR_OK) return s;
  if (op < TSQR_OP_DIRECT || op > TSQR_OP_SVD_VALUES) return TSQR_ERR_ARG;
  const int prec = (opts && op_takes_prec(op)) ? opts->prec : 0;
  Plan P;
  int chunks = 1;
  int rc = op == TSQR_OP_DIRECT_HOST
               ? make_host_plan(m, n, esz, opts ? opts->block_rows : 0, opts ? opts->tree_fanout : 0, &P, &chunks,
                                prec, device_sms())
               : make_plan(m, n, esz, opts ? opts->block_rows : 0, opts ? opts->tree_fanout : 0, &P, prec,
                           device_sms());
  if (rc != TSQR_OK) return static_cast<tsqr_status>(rc);
  std::memset(info, 0, sizeof(*info));
  info->block_rows = P.levels[0].b;
  info->blocks = P.levels[0].p;
  info->tiles_per_block = P.levels[0].kt;
  info->tree_levels = static_cast<int32_t>(P.levels.size()) - 1;
  info->tree_fanout = P.levels.size() > 1 ? static_cast<int32_t>(P.levels[1].b / n) : 0;
  info->prec = P.prec;
  const bool q_pass = op == TSQR_OP_DIRECT || op == TSQR_OP_SVD || op == TSQR_OP_DIRECT_HOST;
  info->step3_tensor = (q_pass && (P.tc3 || P.oz3)) ? 1 : 0;
  return TSQR_OK;
}

tsqr_status tsqr_read_status(const void* work, void* stream) {
  if (!work) return TSQR_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t h = 0;
  if (cudaMemcpyAsync(&h, work, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return TSQR_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return TSQR_ERR_CUDA;
  return static_cast<tsqr_status>(h);
}

tsqr_status tsqr_workspace_size(int32_t op, int64_t m, int64_t n, int32_t dtype, const tsqr_opts* opts,
                                size_t* bytes) {
  if (!bytes) return TSQR_ERR_ARG;
  const int esz = esz_of(dtype);
  if (esz == 0) return TSQR_ERR_ARG;
  tsqr_status s = check_opts(opts);
  if (s != TSQR_OK) return s;
  if (op == TSQR_OP_ACCURACY) {
    if (n < 1 || n > TSQR_NMAX || m < 1 || !rows_fit(m, n)) return TSQR_ERR_SHAPE;
    *bytes = kHeaderBytes + accuracy_geom(m, static_cast<int>(n)).part_bytes;
    return TSQR_OK;
  }
  if (op < TSQR_OP_DIRECT || op > TSQR_OP_SVD_VALUES) return TSQR_ERR_ARG;
  const int prec = (opts && op_takes_prec(op)) ? opts->prec : 0;
  Plan P;
  int chunks = 1;
  int rc = op == TSQR_OP_DIRECT_HOST
               ? make_host_plan(m, n, esz, opts ? opts->block_rows : 0, opts ? opts->tree_fanout : 0, &P, &chunks,
                                prec, device_sms())
               : make_plan(m, n, esz, opts ? opts->block_rows : 0, opts ? opts->tree_fanout : 0, &P, prec,
                           device_sms());
  if (rc != TSQR_OK) return static_cast<tsqr_status>(rc);
  *bytes = op_bytes(P, op);
  return TSQR_OK;
}

tsqr_status tsqr_direct(const void* A, int64_t m, int64_t n, int64_t lda, int32_t dtype, void* Q, int64_t ldq,
                        double* R, int64_t ldr, void* work, size_t work_bytes, const tsqr_opts* opts,
                        void* stream) {
  tsqr_status s = check_tall(A, m, n, lda, dtype, opts);
  if (s != TSQR_OK) return s;
  if (!Q || !R) return TSQR_ERR_ARG;
  if (ldq != n || ldr != n || !aligned16(Q) || !aligned16(R)) return TSQR_ERR_ALIGN;
  const int esz = esz_of(dtype);
  if (overlaps(A, (size_t)m * n * esz, Q, (size_t)m * n * esz)) return TSQR_ERR_ARG;
  Plan P;
  int rc = make_plan(m, n, esz, opts ? opts->block_rows : 0, opts ? opts->tree_fanout : 0, &P,
                     opts ? opts->prec : 0, device_sms());
  if (rc != TSQR_OK) return static_cast<tsqr_status>(rc);
  if (!work || work_bytes < P.bytes || !aligned16(work)) return TSQR_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s = run_direct(P, A, Q, R, ldr, work, st, opts, [](double*, cudaStream_t) { return TSQR_OK; });
  if (s != TSQR_OK) return s;
  return finish(work, opts, st);
}

tsqr_status tsqr_direct_host(const void* A, int64_t m, int64_t n, int32_t dtype, void* Q, double* R,
                             void* dbuf, void* work, size_t work_bytes, const tsqr_opts* opts,
                             void* stream, void* copy_stream) {
  if (!A || !Q || !R || !dbuf || esz_of(dtype) == 0) return TSQR_ERR_ARG;
  if (stream == copy_stream) return TSQR_ERR_ARG;
  tsqr_status s = check_opts(opts);
  if (s != TSQR_OK) return s;
  if (n < 1 || n > TSQR_NMAX || m < n || !rows_fit(m, n)) return TSQR_ERR_SHAPE;
  if (!aligned16(dbuf)) return TSQR_ERR_ALIGN;
  const int esz = esz_of(dtype);
  if (overlaps(A, (size_t)m * n * esz, Q, (size_t)m * n * esz)) return TSQR_ERR_ARG;
  Plan P;
  int chunks = 1;
  int rc = make_host_plan(m, n, esz, opts ? opts->block_rows : 0, opts ? opts->tree_fanout : 0, &P, &chunks,
                          opts ? opts->prec : 0, device_sms());
  if (rc != TSQR_OK) return static_cast<tsqr_status>(rc);
  if (!work || work_bytes < P.bytes || !aligned16(work)) return TSQR_ERR_WORKSPACE;
  if (overlaps(dbuf, (size_t)m * n * esz, work, P.bytes)) return TSQR_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s = run_direct_host(P, chunks, static_cast<const char*>(A), static_cast<char*>(Q), R, static_cast<char*>(dbuf),
                      work, st, static_cast<cudaStream_t>(copy_stream));
  if (s != TSQR_OK) return s;
  return finish(work, opts, st);
}

tsqr_status tsqr_svd(const void* A, int64_t m, int64_t n, int64_t lda, int32_t dtype, void* U, int64_t ldu,
                     double* S, double* V, int64_t ldv, void* work, size_t work_bytes, const tsqr_opts* opts,
                     void* stream) {
  tsqr_status s = check_tall(A, m, n, lda, dtype, opts);
  if (s != TSQR_OK) return s;
  if (!U || !S || !V) return TSQR_ERR_ARG;
  if (ldu != n || ldv != n || !aligned16(U) || !aligned16(S) || !aligned16(V)) return TSQR_ERR_ALIGN;
  const int esz = esz_of(dtype);
  if (overlaps(A, (size_t)m * n * esz, U, (size_t)m * n * esz)) return TSQR_ERR_ARG;
  Plan P;
  TSQR_TRY(plan_for(TSQR_OP_SVD, m, n, dtype, opts, work_bytes, work, &P));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* Rt = reinterpret_cast<double*>(at(work, P.off_small));
  int32_t* status = status_ptr(work);
  const int ni = static_cast<int>(n);
  TSQR_TRY(run_direct(P, A, U, Rt, n, work, st, opts, [&](double* ctop, cudaStream_t ts) {
    return launch_jacobi_svd(Rt, n, ni, ctop, S, V, ldv, status, ts) == cudaSuccess ? TSQR_OK : TSQR_ERR_CUDA;
  }));
  return finish(work, opts, st);
}

tsqr_status tsqr_r(const void* A, int64_t m, int64_t n, int64_t lda, int32_t dtype, double* R, int64_t ldr,
                   void* work, size_t work_bytes, const tsqr_opts* opts, void* stream) {
  tsqr_status s = check_tall(A, m, n, lda, dtype, opts);
  if (s != TSQR_OK) return s;
  if (!R) return TSQR_ERR_ARG;
  if (ldr != n || !aligned16(R)) return TSQR_ERR_ALIGN;
  Plan P;
  TSQR_TRY(plan_for(TSQR_OP_R, m, n, dtype, opts, work_bytes, work, &P));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TSQR_CUDA(cudaMemsetAsync(status_ptr(work), 0, sizeof(int32_t), st));
  // Sec. II-B: Steps 1-2 keep only the R factors; the top R is sign-normalised
  TSQR_TRY(run_r_only(P, esz_of(dtype), A, R, work, st));
  return finish(work, opts, st);
}

tsqr_status tsqr_svd_values(const void* A, int64_t m, int64_t n, int64_t lda, int32_t dtype, double* S, double* V,
                            int64_t ldv, void* work, size_t work_bytes, const tsqr_opts* opts, void* stream) {
  tsqr_status s = check_tall(A, m, n, lda, dtype, opts);
  if (s != TSQR_OK) return s;
  if (!S) return TSQR_ERR_ARG;
  if ((V && ldv != n) || !aligned16(S) || !aligned16_or_null(V)) return TSQR_ERR_ALIGN;
  Plan P;
  TSQR_TRY(plan_for(TSQR_OP_SVD_VALUES, m, n, dtype, opts, work_bytes, work, &P));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t* status = status_ptr(work);
  const size_t nn = (size_t)n * n;
  double* Rt = reinterpret_cast<double*>(at(work, P.off_small));
  double* Vt = V ? V : Rt + nn;  // V not wanted: a scratch slot takes it
  double* ctop = reinterpret_cast<double*>(at(work, P.off_ctop));
  TSQR_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  // Sec. III-B: the singular values of A are those of R (Steps 1-2 + SVD of R)
  TSQR_TRY(run_r_only(P, esz_of(dtype), A, Rt, work, st));
  TSQR_CUDA(launch_jacobi_svd(Rt, n, static_cast<int>(n), ctop, S, Vt, n, status, st));
  return finish(work, opts, st);
}

tsqr_status cholqr(const void* A, int64_t m, int64_t n, int64_t lda, int32_t dtype, void* Q, int64_t ldq,
                   double* R, int64_t ldr, int32_t refine_steps, void* work, size_t work_bytes,
                   const tsqr_opts* opts, void* stream) {
  tsqr_status s = check_tall(A, m, n, lda, dtype, opts);
  if (s != TSQR_OK) return s;
  if (!Q || !R || refine_steps < 0) return TSQR_ERR_ARG;
  if (ldq != n || ldr != n || !aligned16(Q) || !aligned16(R)) return TSQR_ERR_ALIGN;
  const int esz = esz_of(dtype);
  if (overlaps(A, (size_t)m * n * esz, Q, (size_t)m * n * esz)) return TSQR_ERR_ARG;
  Plan P;
  TSQR_TRY(plan_for(TSQR_OP_CHOLQR, m, n, dtype, opts, work_bytes, work, &P));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t* status = status_ptr(work);
  const size_t nn = (size_t)n * n;
  double* part = reinterpret_cast<double*>(at(work, P.off_part));
  double* G = reinterpret_cast<double*>(at(work, P.off_gsmall));
  double* R1 = G + nn;
  double* R2 = G + 2 * nn;
  double* Rinv = G + 3 * nn;
  const int ni = static_cast<int>(n);
  TSQR_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  // Sec. II-A: A^T A = sum_p A_p^T A_p, Cholesky, then Q = A R^{-1} (Sec. II-C)
  TSQR_CUDA(launch_gram(esz, A, A, m, ni, part, G, status, st));
  TSQR_CUDA(launch_chol_inv(G, ni, R1, Rinv, status, st));
  TSQR_TRY(rowmul(P, A, Rinv, nullptr, nullptr, Q, status, st));
  for (int r = 0; r < refine_steps; ++r) {  // iterative refinement: repeat on the computed Q
    TSQR_CUDA(launch_gram(esz, Q, Q, m, ni, part, G, status, st));
    TSQR_CUDA(launch_chol_inv(G, ni, R2, Rinv, status, st));
    TSQR_TRY(rowmul(P, Q, Rinv, nullptr, nullptr, Q, status, st));
    TSQR_CUDA(launch_tri_mul(R2, R1, ni, R1, n, st));
  }
  TSQR_TRY(copy_r(R, ldr, R1, n, st));
  return finish(work, opts, st);
}

tsqr_status tsqr_indirect_refine(const void* A, int64_t m, int64_t n, int64_t lda, int32_t dtype, void* Q,
                                 int64_t ldq, double* R, int64_t ldr, int32_t refine_steps, void* work,
                                 size_t work_bytes, const tsqr_opts* opts, void* stream) {
  tsqr_status s = check_tall(A, m, n, lda, dtype, opts);
  if (s != TSQR_OK) return s;
  if (!Q || !R || refine_steps < 0) return TSQR_ERR_ARG;
  if (ldq != n || ldr != n || !aligned16(Q) || !aligned16(R)) return TSQR_ERR_ALIGN;
  const int esz = esz_of(dtype);
  if (overlaps(A, (size_t)m * n * esz, Q, (size_t)m * n * esz)) return TSQR_ERR_ARG;
  Plan P;
  TSQR_TRY(plan_for(TSQR_OP_INDIRECT, m, n, dtype, opts, work_bytes, work, &P));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t* status = status_ptr(work);
  const size_t nn = (size_t)n * n;
  double* R1 = reinterpret_cast<double*>(at(work, P.off_small));
  double* R2 = R1 + nn;
  double* Rinv = R1 + 2 * nn;
  const int ni = static_cast<int>(n);
  TSQR_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  // Sec. II-B: R from the TSQR reduction; Sec. II-C: Q = A R^{-1}
  TSQR_TRY(run_r_only(P, esz, A, R1, work, st));
  TSQR_CUDA(launch_rinv(R1, n, ni, Rinv, status, st));
  TSQR_TRY(rowmul(P, A, Rinv, nullptr, nullptr, Q, status, st));
  for (int r = 0; r < refine_steps; ++r) {  // refinement: repeat on the computed Q
    TSQR_TRY(run_r_only(P, esz, Q, R2, work, st));
    TSQR_CUDA(launch_rinv(R2, n, ni, Rinv, status, st));
    TSQR_TRY(rowmul(P, Q, Rinv, nullptr, nullptr, Q, status, st));
    TSQR_CUDA(launch_tri_mul(R2, R1, ni, R1, n, st));
  }
  TSQR_TRY(copy_r(R, ldr, R1, n, st));
  return finish(work, opts, st);
}

tsqr_status tsqr_accuracy(const void* A, const void* Q, const double* R, int64_t m, int64_t n, int32_t dtype,
                          double* out, void* work, size_t work_bytes, void* stream) {
  const int esz = esz_of(dtype);
  if (!Q || !out || esz == 0 || (A == nullptr) != (R == nullptr)) return TSQR_ERR_ARG;
  if (n < 1 || n > TSQR_NMAX || m < 1 || !rows_fit(m, n)) return TSQR_ERR_SHAPE;
  if (!aligned16(Q) || !aligned16(out) || !aligned16_or_null(A) || !aligned16_or_null(R)) return TSQR_ERR_ALIGN;
  const size_t need = kHeaderBytes + accuracy_geom(m, static_cast<int>(n)).part_bytes;
  if (!work || !aligned16(work) || work_bytes < need) return TSQR_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  TSQR_CUDA(cudaMemsetAsync(status_ptr(work), 0, sizeof(int32_t), st));
  double* part = reinterpret_cast<double*>(at(work, kHeaderBytes));
  TSQR_CUDA(launch_accuracy(esz, Q, A, R, m, static_cast<int>(n), part, out, st));
  return finish(work, nullptr, st);
}

tsqr_status tsqr_backward(const void* Q, const double* R, const void* dQ, const double* dR, int64_t m, int64_t n,
                          int32_t dtype, void* dA, void* work, size_t work_bytes, const tsqr_opts* opts,
                          void* stream) {
  tsqr_status s = check_tall(Q, m, n, n, dtype, opts);
  if (s != TSQR_OK) return s;
  if (!R || !dA) return TSQR_ERR_ARG;
  if (!aligned16(dA) || !aligned16_or_null(dQ) || !aligned16(R) || !aligned16_or_null(dR)) return TSQR_ERR_ALIGN;
  Plan P;
  TSQR_TRY(plan_for(TSQR_OP_BACKWARD, m, n, dtype, opts, work_bytes, work, &P));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int32_t* status = status_ptr(work);
  const size_t nn = (size_t)n * n;
  const int esz = esz_of(dtype);
  double* part = reinterpret_cast<double*>(at(work, P.off_part));
  double* G = reinterpret_cast<double*>(at(work, P.off_gsmall));
  double* M1 = G + nn;
  double* M2 = G + 2 * nn;
  const int ni = static_cast<int>(n);
  TSQR_CUDA(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
  if (dQ) TSQR_CUDA(launch_gram(esz, dQ, Q, m, ni, part, G, status, st, esz == 4));  // G = dQ^T Q
  TSQR_CUDA(launch_bwd_prep(R, dR, dQ ? G : nullptr, ni, M1, M2, status, st));
  // dA = (dQ + Q copyltu(M)) R^{-T} = dQ R^{-T} + Q (copyltu(M) R^{-T})
  TSQR_TRY(rowmul(P, dQ, M1, Q, M2, dA, status, st));
  return finish(work, opts, st);
}

}  // extern "C"
