// small.cuh -- single-CTA kernels on n x n binary64 matrices.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tsqr {

// Sign normalisation of the top R (Sec. II-A uniqueness: diag(R) >= 0):
// D = diag(sign(R_jj)), sign(0) = +1; Rout = D Rraw (lower part zeroed),
// Ctop = D.  Flags TSQR_ERR_NONFINITE if Rraw holds a NaN or Inf.
cudaError_t launch_sign_fix(const double* Rraw, int n, double* Rout, int64_t ldr, double* Ctop,
                            int32_t* status, cudaStream_t st);

// R = chol(G) (upper) and Rinv = R^{-1}; breakdown -> TSQR_ERR_NOT_SPD.
cudaError_t launch_chol_inv(const double* G, int n, double* R, double* Rinv, int32_t* status, cudaStream_t st);
// Rinv = R^{-1} (R upper, leading dimension ldr); zero diagonal -> SINGULAR.
cudaError_t launch_rinv(const double* R, int64_t ldr, int n, double* Rinv, int32_t* status, cudaStream_t st);
// Rout = R2 R1 (upper triangular); Rout may alias R1.
cudaError_t launch_tri_mul(const double* R2, const double* R1, int n, double* Rout, int64_t ldr, cudaStream_t st);
// Adjoint prep: M1 = R^{-T}, M2 = copyltu(R dR^T - G) R^{-T} (dR, G nullable).
cudaError_t launch_bwd_prep(const double* R, const double* dR, const double* G, int n, double* M1, double* M2,
                            int32_t* status, cudaStream_t st);
// One-sided Jacobi SVD of R (ldr): S (n), V (ldv); Ctop (n x n, holding the
// sign matrix D) becomes D U_R.
cudaError_t launch_jacobi_svd(const double* R, int64_t ldr, int n, double* Ctop, double* S, double* V,
                              int64_t ldv, int32_t* status, cudaStream_t st);

// In place: p blocks of (tau on the diagonal, Gram v_i^T v_j above) -> T_i.
cudaError_t launch_build_t(double* Tst, int64_t p, int n, bool binary32, cudaStream_t st);
// G = sum of the nparts n x n partials in index order (deterministic).
cudaError_t launch_gram_reduce(const double* part, int nparts, int n, double* G, int32_t* status,
                               cudaStream_t st);

}  // namespace tsqr
