// kern_inst.cuh -- instantiates the TSQR kernels for one (storage, compute)
// type pair and seven register tiles (R_i rows x N_i columns per thread, at
// most T_i threads per CTA so that registers x threads <= 64K; N_i = 5 unless
// TSQR_N_i says otherwise); included once per translation unit, which names
// the launchers it wants (TSQR_LOCAL_QR_NAME and TSQR_FORM_Q_NAME,
// TSQR_LOCAL_R_NAME, TSQR_ROWMUL_NAME with TSQR_GRAM_NAME).
// KernelCfg::tile selects the tile.
#pragma once

#include "launch.h"
#include "qr_kernels.cuh"
#include "tall_kernels.cuh"

namespace tsqr {

#ifdef TSQR_LOCAL_QR_NAME
template <int R, int MAXT, int NPC>
static cudaError_t local_qr_R(const KernelCfg& k, const TSQR_S* A, int64_t m, int n, int64_t b, int64_t bt, int kt,
                              int64_t p, TSQR_S* Y, double* Rst, double* Tst, int32_t* status, cudaStream_t st) {
  if (k.NT > MAXT) return cudaErrorInvalidConfiguration;
  // the look-ahead form when the tile is one row group
  auto fn = k.NRG == 1 ? k_local_qr<TSQR_S, TSQR_T, NPC, R, MAXT, true>
                       : k_local_qr<TSQR_S, TSQR_T, NPC, R, MAXT, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem_qr);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)p, k.NT, k.smem_qr, st>>>(A, m, n, (int)b, (int)bt, kt, k.CS, k.NRG, Y, Rst, Tst, status);
  return cudaGetLastError();
}

template <int R, int MAXT, int NPC>
static cudaError_t form_q_R(const KernelCfg& k, const TSQR_S* Y, int64_t m, int n, int64_t b, int64_t bt, int kt,
                            int64_t p, const double* T, const double* C, int64_t cblocks, TSQR_S* Q,
                            int32_t* status, cudaStream_t st) {
  if (k.NT > MAXT) return cudaErrorInvalidConfiguration;
  auto fn = k_form_q<TSQR_S, TSQR_T, NPC, R, MAXT>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem_fq);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)p, k.NT, k.smem_fq, st>>>(Y, m, n, (int)b, (int)bt, kt, k.fq_rows, k.CS, k.NRG, k.skew, T, C,
                                           cblocks, Q, status);
  return cudaGetLastError();
}

cudaError_t TSQR_LOCAL_QR_NAME(const KernelCfg& k, const void* A, int64_t m, int n, int64_t b, int64_t bt, int kt,
                               int64_t p, void* Y, double* Rst, double* Tst, int32_t* status, cudaStream_t st) {
  const TSQR_S* a = static_cast<const TSQR_S*>(A);
  TSQR_S* y = static_cast<TSQR_S*>(Y);
  switch (k.tile) {
    case 0: return local_qr_R<TSQR_R0, TSQR_T0, kNpc>(k, a, m, n, b, bt, kt, p, y, Rst, Tst, status, st);
    case 1: return local_qr_R<TSQR_R1, TSQR_T1, kNpc>(k, a, m, n, b, bt, kt, p, y, Rst, Tst, status, st);
    case 2: return local_qr_R<TSQR_R2, TSQR_T2, kNpc>(k, a, m, n, b, bt, kt, p, y, Rst, Tst, status, st);
    case 3: return local_qr_R<TSQR_R3, TSQR_T3, kNpc>(k, a, m, n, b, bt, kt, p, y, Rst, Tst, status, st);
    case 4: return local_qr_R<TSQR_R4, TSQR_T4, kNpc>(k, a, m, n, b, bt, kt, p, y, Rst, Tst, status, st);
    case 5: return local_qr_R<TSQR_R5, TSQR_T5, TSQR_N5>(k, a, m, n, b, bt, kt, p, y, Rst, Tst, status, st);
    case 6: return local_qr_R<TSQR_R6, TSQR_T6, TSQR_N6>(k, a, m, n, b, bt, kt, p, y, Rst, Tst, status, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t TSQR_FORM_Q_NAME(const KernelCfg& k, const void* Y, int64_t m, int n, int64_t b, int64_t bt, int kt,
                             int64_t p, const double* T, const double* C, int64_t cblocks, void* Q,
                             int32_t* status, cudaStream_t st) {
  const TSQR_S* y = static_cast<const TSQR_S*>(Y);
  TSQR_S* q = static_cast<TSQR_S*>(Q);
  switch (k.tile) {
    case 0: return form_q_R<TSQR_R0, TSQR_T0, kNpc>(k, y, m, n, b, bt, kt, p, T, C, cblocks, q, status, st);
    case 1: return form_q_R<TSQR_R1, TSQR_T1, kNpc>(k, y, m, n, b, bt, kt, p, T, C, cblocks, q, status, st);
    case 2: return form_q_R<TSQR_R2, TSQR_T2, kNpc>(k, y, m, n, b, bt, kt, p, T, C, cblocks, q, status, st);
    case 3: return form_q_R<TSQR_R3, TSQR_T3, kNpc>(k, y, m, n, b, bt, kt, p, T, C, cblocks, q, status, st);
    case 4: return form_q_R<TSQR_R4, TSQR_T4, kNpc>(k, y, m, n, b, bt, kt, p, T, C, cblocks, q, status, st);
    case 5: return form_q_R<TSQR_R5, TSQR_T5, TSQR_N5>(k, y, m, n, b, bt, kt, p, T, C, cblocks, q, status, st);
    case 6: return form_q_R<TSQR_R6, TSQR_T6, TSQR_N6>(k, y, m, n, b, bt, kt, p, T, C, cblocks, q, status, st);
    default: return cudaErrorInvalidValue;
  }
}
#endif  // TSQR_LOCAL_QR_NAME

#ifdef TSQR_LOCAL_R_NAME
// R-only local QR (Y, T and the Gram dot products left out) for the
// one-row-group tiles (the look-ahead loop); other tiles take the general
// kernel with Y == NULL.
template <int R, int MAXT, int NPC>
static cudaError_t local_r_R(const KernelCfg& k, const TSQR_S* A, int64_t m, int n, int64_t b, int64_t bt, int kt,
                             int64_t p, double* Rst, int32_t* status, cudaStream_t st) {
  if (k.NT > MAXT || k.NRG != 1) return cudaErrorInvalidConfiguration;
  auto fn = k_local_qr<TSQR_S, TSQR_T, NPC, R, MAXT, true, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem_qr);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)p, k.NT, k.smem_qr, st>>>(A, m, n, (int)b, (int)bt, kt, k.CS, k.NRG, nullptr, Rst, nullptr,
                                           status);
  return cudaGetLastError();
}

cudaError_t TSQR_LOCAL_R_NAME(const KernelCfg& k, const void* A, int64_t m, int n, int64_t b, int64_t bt, int kt,
                              int64_t p, double* Rst, int32_t* status, cudaStream_t st) {
  const TSQR_S* a = static_cast<const TSQR_S*>(A);
  switch (k.tile) {
    case 0: return local_r_R<TSQR_R0, TSQR_T0, kNpc>(k, a, m, n, b, bt, kt, p, Rst, status, st);
    case 1: return local_r_R<TSQR_R1, TSQR_T1, kNpc>(k, a, m, n, b, bt, kt, p, Rst, status, st);
    case 2: return local_r_R<TSQR_R2, TSQR_T2, kNpc>(k, a, m, n, b, bt, kt, p, Rst, status, st);
    case 3: return local_r_R<TSQR_R3, TSQR_T3, kNpc>(k, a, m, n, b, bt, kt, p, Rst, status, st);
    case 4: return local_r_R<TSQR_R4, TSQR_T4, kNpc>(k, a, m, n, b, bt, kt, p, Rst, status, st);
    case 5: return local_r_R<TSQR_R5, TSQR_T5, TSQR_N5>(k, a, m, n, b, bt, kt, p, Rst, status, st);
    case 6: return local_r_R<TSQR_R6, TSQR_T6, TSQR_N6>(k, a, m, n, b, bt, kt, p, Rst, status, st);
    default: return cudaErrorInvalidValue;
  }
}
#endif  // TSQR_LOCAL_R_NAME

#ifdef TSQR_LOCAL_QR_NOGRAM_NAME
// Y, R and tau without the Gram dot products (the same kernel instantiation
// as the R-only form, given Y and the T slots): the one-row-group tiles.
template <int R, int MAXT, int NPC>
static cudaError_t local_qr_ng_R(const KernelCfg& k, const TSQR_S* A, int64_t m, int n, int64_t b, int64_t bt, int kt,
                                 int64_t p, TSQR_S* Y, double* Rst, double* Tst, int32_t* status, cudaStream_t st) {
  if (k.NT > MAXT || k.NRG != 1) return cudaErrorInvalidConfiguration;
  auto fn = k_local_qr<TSQR_S, TSQR_T, NPC, R, MAXT, true, false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem_qr);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)p, k.NT, k.smem_qr, st>>>(A, m, n, (int)b, (int)bt, kt, k.CS, k.NRG, Y, Rst, Tst, status);
  return cudaGetLastError();
}

cudaError_t TSQR_LOCAL_QR_NOGRAM_NAME(const KernelCfg& k, const void* A, int64_t m, int n, int64_t b, int64_t bt,
                                      int kt, int64_t p, void* Y, double* Rst, double* Tst, int32_t* status,
                                      cudaStream_t st) {
  const TSQR_S* a = static_cast<const TSQR_S*>(A);
  TSQR_S* y = static_cast<TSQR_S*>(Y);
  switch (k.tile) {
    case 0: return local_qr_ng_R<TSQR_R0, TSQR_T0, kNpc>(k, a, m, n, b, bt, kt, p, y, Rst, Tst, status, st);
    case 1: return local_qr_ng_R<TSQR_R1, TSQR_T1, kNpc>(k, a, m, n, b, bt, kt, p, y, Rst, Tst, status, st);
    case 2: return local_qr_ng_R<TSQR_R2, TSQR_T2, kNpc>(k, a, m, n, b, bt, kt, p, y, Rst, Tst, status, st);
    case 3: return local_qr_ng_R<TSQR_R3, TSQR_T3, kNpc>(k, a, m, n, b, bt, kt, p, y, Rst, Tst, status, st);
    case 4: return local_qr_ng_R<TSQR_R4, TSQR_T4, kNpc>(k, a, m, n, b, bt, kt, p, y, Rst, Tst, status, st);
    case 5: return local_qr_ng_R<TSQR_R5, TSQR_T5, TSQR_N5>(k, a, m, n, b, bt, kt, p, y, Rst, Tst, status, st);
    case 6: return local_qr_ng_R<TSQR_R6, TSQR_T6, TSQR_N6>(k, a, m, n, b, bt, kt, p, y, Rst, Tst, status, st);
    default: return cudaErrorInvalidValue;
  }
}
#endif  // TSQR_LOCAL_QR_NOGRAM_NAME

#ifdef TSQR_ROWMUL_NAME
template <int R, int MAXT, int NPC>
static cudaError_t rowmul_R(const KernelCfg& k, const TSQR_S* X, const double* M1, const TSQR_S* Y,
                            const double* M2, int64_t m, int n, int64_t b, int64_t p, TSQR_S* out,
                            int32_t* status, cudaStream_t st) {
  if (k.NT > MAXT) return cudaErrorInvalidConfiguration;
  auto fn = k_rowmul<TSQR_S, TSQR_T, NPC, R, MAXT>;
  const size_t smem = k.smem_rm;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)p, k.NT, smem, st>>>(X, M1, Y, M2, m, n, (int)b, k.rm_rows, k.CS, k.NRG, k.skew, out, status);
  return cudaGetLastError();
}

cudaError_t TSQR_ROWMUL_NAME(const KernelCfg& k, const void* X, const double* M1, const void* Y, const double* M2,
                             int64_t m, int n, int64_t b, int64_t p, void* out, int32_t* status,
                             cudaStream_t st) {
  const TSQR_S* x = static_cast<const TSQR_S*>(X);
  const TSQR_S* y = static_cast<const TSQR_S*>(Y);
  TSQR_S* o = static_cast<TSQR_S*>(out);
  switch (k.tile) {
    case 0: return rowmul_R<TSQR_R0, TSQR_T0, kNpc>(k, x, M1, y, M2, m, n, b, p, o, status, st);
    case 1: return rowmul_R<TSQR_R1, TSQR_T1, kNpc>(k, x, M1, y, M2, m, n, b, p, o, status, st);
    case 2: return rowmul_R<TSQR_R2, TSQR_T2, kNpc>(k, x, M1, y, M2, m, n, b, p, o, status, st);
    case 3: return rowmul_R<TSQR_R3, TSQR_T3, kNpc>(k, x, M1, y, M2, m, n, b, p, o, status, st);
    case 4: return rowmul_R<TSQR_R4, TSQR_T4, kNpc>(k, x, M1, y, M2, m, n, b, p, o, status, st);
    case 5: return rowmul_R<TSQR_R5, TSQR_T5, TSQR_N5>(k, x, M1, y, M2, m, n, b, p, o, status, st);
    case 6: return rowmul_R<TSQR_R6, TSQR_T6, TSQR_N6>(k, x, M1, y, M2, m, n, b, p, o, status, st);
    default: return cudaErrorInvalidValue;
  }
}

// acc_storage: accumulate each CTA's partial Gram in the storage type (the
// adjoint of binary32 data); else in binary64.
cudaError_t TSQR_GRAM_NAME(const void* X, const void* Y, int64_t m, int n, int chunk, int grid, int nt, int tile,
                           bool acc_storage, double* part, int32_t* status, cudaStream_t st) {
  const size_t smem = 2 * align_up((size_t)chunk * n * sizeof(TSQR_S), 16) + 16;
  auto fn = acc_storage ? (tile == 5 ? k_gram<TSQR_S, 5, TSQR_S> : k_gram<TSQR_S, 4, TSQR_S>)
                        : (tile == 5 ? k_gram<TSQR_S, 5, double> : k_gram<TSQR_S, 4, double>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, nt, smem, st>>>(static_cast<const TSQR_S*>(X), static_cast<const TSQR_S*>(Y), m, n, chunk, part,
                             status);
  return cudaGetLastError();
}

#endif  // TSQR_ROWMUL_NAME

}  // namespace tsqr
