// small.cu -- single-CTA binary64 kernels on n x n matrices (n <= 100).
// See small.cuh for the contract of each launcher.
#include <cfloat>

#include "device.cuh"
#include "small.cuh"

namespace tsqr {

// ---------------------------------------------------------------------------
__global__ void k_sign_fix(const double* __restrict__ Rraw, int n, double* __restrict__ Rout, int64_t ldr,
                           double* __restrict__ Ctop, int32_t* status) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, k = idx % n;
    const double rik = Rraw[idx];
    if (!isfinite(rik)) set_status(status, TSQR_ERR_NONFINITE);
    const double d = Rraw[i * n + i] < 0.0 ? -1.0 : 1.0;
    Rout[i * ldr + k] = (k >= i) ? d * rik : 0.0;
    Ctop[idx] = (i == k) ? d : 0.0;
  }
}

cudaError_t launch_sign_fix(const double* Rraw, int n, double* Rout, int64_t ldr, double* Ctop, int32_t* status,
                            cudaStream_t st) {
  k_sign_fix<<<1, 256, 0, st>>>(Rraw, n, Rout, ldr, Ctop, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Inverse of the upper-triangular R (smem copy `r`, n x n) into `x`, column
// by column (one thread per column, back substitution).  Returns false (all
// threads) if a diagonal entry is zero or not finite.
__device__ bool cta_upper_inverse(const double* r, int n, double* x) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    if (r[j * n + j] == 0.0 || !isfinite(r[j * n + j])) bad = 1;
  __syncthreads();
  if (bad) return false;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    for (int i = n - 1; i >= 0; --i) {
      double v;
      if (i > c) {
        v = 0.0;
      } else {
        double s = (i == c) ? 1.0 : 0.0;
        for (int k = i + 1; k <= c; ++k) s = fma(-r[i * n + k], x[k * n + c], s);
        v = s / r[i * n + i];
      }
      x[i * n + c] = v;
    }
  }
  __syncthreads();
  return true;
}

// Cholesky QR's small step (Sec. II-A): R = chol(G) (upper, G = R^T R), and
// Rinv = R^{-1} for Q = A R^{-1} (Sec. II-C computes the inverse of R and
// multiplies by A).  Breakdown -> TSQR_ERR_NOT_SPD.
__global__ void k_chol_inv(const double* __restrict__ G, int n, double* __restrict__ R, double* __restrict__ Rinv,
                           int32_t* status) {
  extern __shared__ __align__(16) double sm[];
  double* a = sm;          // n x n: G, then R in its upper triangle
  double* x = sm + n * n;  // n x n: R^{-1}
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) a[idx] = G[idx];
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double s = a[j * n + j];
      for (int k = 0; k < j; ++k) s = fma(-a[k * n + j], a[k * n + j], s);
      if (!(s > 0.0) || !isfinite(s)) {
        fail = 1;
      } else {
        a[j * n + j] = sqrt(s);
      }
    }
    __syncthreads();
    if (fail) break;
    const double rjj = a[j * n + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
      double t = a[j * n + i];
      for (int k = 0; k < j; ++k) t = fma(-a[k * n + j], a[k * n + i], t);
      a[j * n + i] = t / rjj;
    }
    __syncthreads();
  }
  if (fail) {
    if (threadIdx.x == 0) set_status(status, TSQR_ERR_NOT_SPD);
    return;
  }
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, k = idx % n;
    if (k < i) a[idx] = 0.0;
  }
  __syncthreads();
  if (!cta_upper_inverse(a, n, x)) {
    if (threadIdx.x == 0) set_status(status, TSQR_ERR_NOT_SPD);
    return;
  }
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    R[idx] = a[idx];
    Rinv[idx] = x[idx];
  }
}

cudaError_t launch_chol_inv(const double* G, int n, double* R, double* Rinv, int32_t* status, cudaStream_t st) {
  const size_t smem = 2 * (size_t)n * n * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_chol_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_chol_inv<<<1, 128, smem, st>>>(G, n, R, Rinv, status);
  return cudaGetLastError();
}

// Rinv = R^{-1} of an upper-triangular R (ldr); zero diagonal -> SINGULAR.
__global__ void k_rinv(const double* __restrict__ R, int64_t ldr, int n, double* __restrict__ Rinv,
                       int32_t* status) {
  extern __shared__ __align__(16) double sm[];
  double* a = sm;
  double* x = sm + n * n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, k = idx % n;
    a[idx] = (k >= i) ? R[i * ldr + k] : 0.0;
  }
  __syncthreads();
  if (!cta_upper_inverse(a, n, x)) {
    if (threadIdx.x == 0) set_status(status, TSQR_ERR_SINGULAR);
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) Rinv[idx] = 0.0;
    return;
  }
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) Rinv[idx] = x[idx];
}

cudaError_t launch_rinv(const double* R, int64_t ldr, int n, double* Rinv, int32_t* status, cudaStream_t st) {
  const size_t smem = 2 * (size_t)n * n * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_rinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_rinv<<<1, 128, smem, st>>>(R, ldr, n, Rinv, status);
  return cudaGetLastError();
}

// Rout = R2 R1 (both upper triangular; the refinement's R = R2 R1).  Rout may
// alias R1: the product is formed in shared memory first.
__global__ void k_tri_mul(const double* __restrict__ R2, const double* R1, int n, double* Rout, int64_t ldr) {
  extern __shared__ __align__(16) double sm[];
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, k = idx % n;
    double s = 0.0;
    for (int l = i; l <= k; ++l) s = fma(R2[i * n + l], R1[l * n + k], s);
    sm[idx] = (k >= i) ? s : 0.0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) Rout[(idx / n) * ldr + idx % n] = sm[idx];
}

cudaError_t launch_tri_mul(const double* R2, const double* R1, int n, double* Rout, int64_t ldr, cudaStream_t st) {
  const size_t smem = (size_t)n * n * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_tri_mul, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_tri_mul<<<1, 256, smem, st>>>(R2, R1, n, Rout, ldr);
  return cudaGetLastError();
}

// Adjoint's small step: M = R dR^T - G (G = dQ^T Q; dR upper part only; either
// may be NULL), C = copyltu(M) = tril(M) + tril(M,-1)^T, M1 = R^{-T},
// M2 = C R^{-T}.  Then dA = dQ M1 + Q M2.  Zero diagonal -> SINGULAR.
__global__ void k_bwd_prep(const double* __restrict__ R, const double* __restrict__ dR,
                           const double* __restrict__ G, int n, double* __restrict__ M1, double* __restrict__ M2,
                           int32_t* status) {
  extern __shared__ __align__(16) double sm[];
  double* r = sm;              // R (upper)
  double* x = sm + n * n;      // R^{-1}
  double* mm = sm + 2 * n * n; // M, then C
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, k = idx % n;
    r[idx] = (k >= i) ? R[idx] : 0.0;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, j = idx % n;
    double s = 0.0;
    if (dR)
      for (int k = (i > j ? i : j); k < n; ++k) s = fma(r[i * n + k], dR[j * n + k], s);  // dR upper: k >= j
    if (G) s -= G[idx];
    mm[idx] = s;
  }
  __syncthreads();
  const bool ok = cta_upper_inverse(r, n, x);
  if (!ok) {
    if (threadIdx.x == 0) set_status(status, TSQR_ERR_SINGULAR);
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      M1[idx] = 0.0;
      M2[idx] = 0.0;
    }
    return;
  }
  // C = copyltu(M) in place: read both triangles first
  double cvals[40];
  const int per = (n * n + blockDim.x - 1) / blockDim.x;  // <= 40 for n <= 100, blockDim >= 256
  for (int t = 0; t < per; ++t) {
    const int idx = threadIdx.x + t * blockDim.x;
    if (idx < n * n) {
      const int i = idx / n, j = idx % n;
      cvals[t] = (i >= j) ? mm[i * n + j] : mm[j * n + i];
    }
  }
  __syncthreads();
  for (int t = 0; t < per; ++t) {
    const int idx = threadIdx.x + t * blockDim.x;
    if (idx < n * n) mm[idx] = cvals[t];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int k = idx / n, c = idx % n;
    M1[idx] = x[c * n + k];  // R^{-T}
    double s = 0.0;
    for (int l = c; l < n; ++l) s = fma(mm[k * n + l], x[c * n + l], s);  // (C R^{-T})_{kc}
    M2[idx] = s;
  }
}

cudaError_t launch_bwd_prep(const double* R, const double* dR, const double* G, int n, double* M1, double* M2,
                            int32_t* status, cudaStream_t st) {
  const size_t smem = 3 * (size_t)n * n * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_bwd_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_bwd_prep<<<1, 256, smem, st>>>(R, dR, G, n, M1, M2, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// SVD of the n x n R (Sec. III-B, SVD paragraph) by one-sided (Hestenes)
// Jacobi in binary64, applied to X = R^T: the columns of X (the rows of R)
// are rotated pairwise until mutually orthogonal, X J = U_X diag(S), so
// R = J diag(S) U_X^T: U_R = J (the accumulated rotations) and V = U_X
// (the normalised columns of X).  Rotating R^T rather than R takes fewer
// sweeps (the rows of a triangular factor are graded; 10-12 instead of 15-32
// sweeps at n = 25..100, kappa up to 1e15).  S is sorted descending and each
// (u_j, v_j) signed so that the largest-|.| entry of v_j is positive (lowest
// index wins a tie).  The top coefficient Ctop, holding the sign matrix D on
// entry, becomes D U_R, so that Step 3 writes U = Q U_R directly.
//
// One cluster of kJacCl CTAs (kJacCl SMs' binary64 units); CTA r holds rows
// [r nr, (r + 1) nr) of X and J.  The pairs of a round follow the
// round-robin (circle) tournament: position 0 is fixed, positions 1..np-1
// rotate by one per round, pair k is (position k, position np-1-k).  A round:
//   A. one thread per pair forms the partial dot products (x_p.x_p, x_q.x_q,
//      x_p.x_q) over the CTA's rows and stores them into every CTA's shared
//      memory (distributed shared memory), double-buffered by round parity;
//   B. one cluster barrier; each CTA sums the kJacCl partials in rank order
//      -- the same values in the same order in every CTA, so every CTA takes
//      bit-identical rotation decisions and (c, s) -- one thread per pair;
//   C. every thread rotates (pair, row) items of its CTA's rows of X and J.
// The binary64 unit serves whole warps, so one thread per pair spends a warp
// instruction on 32 pairs where a warp per pair would spend it on one.
// Every CTA runs the same number of cluster barriers (the convergence test is
// the same in all of them); the last one precedes the exit, so no CTA leaves
// while another still writes into its shared memory.
constexpr int kJacCl = 8;    // CTAs per cluster (portable cluster size)
constexpr int kJacNT = 256;  // threads per CTA

struct JacobiSmem {
  int np, npair, nr, ld;
  size_t x, j, part, fin, pc, ps, d, sv, sg, pp, pq, rank, bytes;
  __host__ __device__ JacobiSmem(int n) {
    np = (n + 1) & ~1;
    npair = np / 2;
    nr = (n + kJacCl - 1) / kJacCl;  // rows per CTA
    ld = nr | 1;                     // odd column stride (thread-per-pair reads spread over banks)
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o += (bytes + 15) / 16 * 16; return at; };
    x = take(sizeof(double) * np * ld);
    j = take(sizeof(double) * np * ld);
    part = take(sizeof(double) * 2 * kJacCl * npair * 3);
    fin = take(sizeof(double) * kJacCl * np * 3);
    pc = take(sizeof(double) * npair);
    ps = take(sizeof(double) * npair);
    d = take(sizeof(double) * nr);
    sv = take(sizeof(double) * np);
    sg = take(sizeof(double) * np);
    pp = take(sizeof(int) * npair);
    pq = take(sizeof(int) * npair);
    rank = take(sizeof(int) * np);
    bytes = o;
  }
};

__global__ void __cluster_dims__(kJacCl, 1, 1) __launch_bounds__(kJacNT)
    k_jacobi_svd(const double* __restrict__ R, int64_t ldr, int n, double* __restrict__ Ctop,
                 double* __restrict__ S, double* __restrict__ V, int64_t ldv, int32_t* status) {
  extern __shared__ __align__(16) unsigned char jsm[];
  const JacobiSmem L(n);
  const int np = L.np, npair = L.npair, nr = L.nr, ld = L.ld;
  double* x = reinterpret_cast<double*>(jsm + L.x);     // column c, local row i at x[c * ld + i]
  double* jm = reinterpret_cast<double*>(jsm + L.j);
  double* part = reinterpret_cast<double*>(jsm + L.part);  // [parity][rank][pair][3]
  double* fin = reinterpret_cast<double*>(jsm + L.fin);    // [rank][column][3]
  double* pc = reinterpret_cast<double*>(jsm + L.pc);
  double* ps = reinterpret_cast<double*>(jsm + L.ps);
  double* d = reinterpret_cast<double*>(jsm + L.d);
  double* sv = reinterpret_cast<double*>(jsm + L.sv);
  double* sgn = reinterpret_cast<double*>(jsm + L.sg);
  int* pp = reinterpret_cast<int*>(jsm + L.pp);
  int* pq = reinterpret_cast<int*>(jsm + L.pq);
  int* rnk = reinterpret_cast<int*>(jsm + L.rank);
  __shared__ int rotated;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int me = static_cast<int>(cluster_ctarank());
  const int r0 = me * nr;
  const int nl = max(0, min(n, r0 + nr) - r0);  // rows held here
  // X(i, c) = R(c, i): local row i of column c
  for (int idx = tid; idx < np * ld; idx += NT) {
    const int c = idx / ld, i = idx - c * ld, g = r0 + i;
    x[idx] = (c < n && i < nl && g >= c) ? R[c * ldr + g] : 0.0;
    jm[idx] = (c < n && i < nl && c == g) ? 1.0 : 0.0;
  }
  for (int i = tid; i < nl; i += NT) d[i] = Ctop[(r0 + i) * n + r0 + i];
  if (tid == 0) rotated = 0;
  cluster_barrier();  // every CTA of the cluster has started (its shared memory exists)
  const double tol = DBL_EPSILON * n;
  const int m1 = np - 1;
  bool converged = false;
  int par = 0;
  for (int sweep = 0; sweep < 60 && !converged; ++sweep) {
    for (int round = 0; round < m1; ++round, par ^= 1) {
      double* pb = part + par * kJacCl * npair * 3;
      // A: partial dots over this CTA's rows, to every CTA
      if (tid < npair) {
        auto col_at = [&](int t) { return t == 0 ? 0 : ((t - 1 - round) % m1 + m1) % m1 + 1; };
        int p = col_at(tid), q = col_at(np - 1 - tid);
        if (p > q) { const int t = p; p = q; q = t; }
        pp[tid] = p;
        pq[tid] = q;
        double al = 0.0, be = 0.0, ga = 0.0;
        if (q < n) {
          const double* xp = x + p * ld;
          const double* xq = x + q * ld;
          for (int i = 0; i < nl; ++i) {
            const double a = xp[i], b = xq[i];
            al = fma(a, a, al);
            be = fma(b, b, be);
            ga = fma(a, b, ga);
          }
        }
        double* slot = pb + (me * npair + tid) * 3;
        for (int k = 0; k < kJacCl; ++k) {
          st_cluster(cluster_map(slot, k), al);
          st_cluster(cluster_map(slot + 1, k), be);
          st_cluster(cluster_map(slot + 2, k), ga);
        }
      }
      cluster_barrier();
      // B: the full dots (rank order) and the rotation, one thread per pair
      if (tid < npair) {
        int q = pq[tid];
        if (q < n) {
          double al = 0.0, be = 0.0, ga = 0.0;
          for (int k = 0; k < kJacCl; ++k) {
            const double* sl = pb + (k * npair + tid) * 3;
            al += sl[0];
            be += sl[1];
            ga += sl[2];
          }
          if (ga != 0.0 && fabs(ga) > tol * sqrt(al * be)) {
            const double zeta = (be - al) / (2.0 * ga);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double c = 1.0 / sqrt(1.0 + t * t);
            pc[tid] = c;
            ps[tid] = c * t;
            rotated = 1;
          } else {
            q = -1;
          }
        } else {
          q = -1;  // the dummy column
        }
        pq[tid] = q;
      }
      __syncthreads();
      // C: rotate columns p and q of this CTA's rows of X and J
      for (int idx = tid; idx < npair * nl; idx += NT) {
        const int k = idx / nl, i = idx - k * nl;
        const int q = pq[k];
        if (q < 0) continue;
        const int p = pp[k];
        const double c = pc[k], s = ps[k];
        const double a = x[p * ld + i], b = x[q * ld + i];
        x[p * ld + i] = c * a - s * b;
        x[q * ld + i] = s * a + c * b;
        const double va = jm[p * ld + i], vb = jm[q * ld + i];
        jm[p * ld + i] = c * va - s * vb;
        jm[q * ld + i] = s * va + c * vb;
      }
      __syncthreads();
    }
    converged = (rotated == 0);  // the same decision in every CTA
    __syncthreads();
    if (tid == 0) rotated = 0;
    __syncthreads();
  }
  if (!converged && tid == 0 && me == 0) set_status(status, TSQR_ERR_NOCONV);
  // column norms and the largest-|.| entry of each column over this CTA's
  // rows (lowest row on ties), to every CTA
  for (int c = tid; c < n; c += NT) {
    double s2 = 0.0, best = -1.0, val = 0.0;
    int bi = 0;
    for (int i = 0; i < nl; ++i) {
      const double v = x[c * ld + i];
      s2 = fma(v, v, s2);
      if (fabs(v) > best) { best = fabs(v); bi = r0 + i; val = v; }
    }
    double* slot = fin + (me * np + c) * 3;
    for (int k = 0; k < kJacCl; ++k) {
      st_cluster(cluster_map(slot, k), s2);
      st_cluster(cluster_map(slot + 1, k), nl > 0 ? best : -1.0);
      st_cluster(cluster_map(slot + 2, k), val);
    }
    (void)bi;
  }
  cluster_barrier();  // the last access to another CTA's shared memory is above
  for (int c = tid; c < n; c += NT) {
    double s2 = 0.0, best = -1.0, val = 0.0;
    for (int k = 0; k < kJacCl; ++k) {  // rank order = row order: strict > keeps the lowest row
      const double* sl = fin + (k * np + c) * 3;
      s2 += sl[0];
      if (sl[1] > best) { best = sl[1]; val = sl[2]; }
    }
    sv[c] = sqrt(s2);
    sgn[c] = val < 0.0 ? -1.0 : 1.0;
  }
  __syncthreads();
  // rank by descending singular value (ties by index)
  for (int c = tid; c < n; c += NT) {
    int r = 0;
    for (int k = 0; k < n; ++k)
      if (sv[k] > sv[c] || (sv[k] == sv[c] && k < c)) ++r;
    rnk[c] = r;
    if (me == 0) S[r] = sv[c];
  }
  __syncthreads();
  // this CTA's rows of V = U_X (signed, normalised) and of D U_R = D J (signed)
  for (int idx = tid; idx < nl * n; idx += NT) {
    const int i = idx / n, c = idx - i * n, g = r0 + i;
    const double inv = sv[c] > 0.0 ? 1.0 / sv[c] : 0.0;
    V[g * ldv + rnk[c]] = sgn[c] * x[c * ld + i] * inv;
    Ctop[g * n + rnk[c]] = d[i] * sgn[c] * jm[c * ld + i];
  }
}

cudaError_t launch_jacobi_svd(const double* R, int64_t ldr, int n, double* Ctop, double* S, double* V,
                              int64_t ldv, int32_t* status, cudaStream_t st) {
  const JacobiSmem L(n);
  cudaError_t e = cudaFuncSetAttribute(k_jacobi_svd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
  if (e != cudaSuccess) return e;
  k_jacobi_svd<<<kJacCl, kJacNT, L.bytes, st>>>(R, ldr, n, Ctop, S, V, ldv, status);
  return cudaGetLastError();
}

// Compact-WY T factors of p row blocks, in place (one warp per block): the
// slot holds tau_j on the diagonal and the Gram entries G(i,j) = v_i^T v_j
// above it; T(j,j) = tau_j and T(i,j) = -tau_j sum_{l=i}^{j-1} T(i,l) G(l,j),
// four columns per pass (H_1 ... H_k = I - Y T Y^T).  Each warp stages the
// upper triangle of its slot in shared memory, packed by columns (entry
// (i, c), i <= c, at c (c + 1) / 2 + i: half the space of a square stage, so
// twice the warps per SM), runs the recursion there in type F and writes it
// back (binary64 slots; F = binary32 for the row blocks of binary32 data,
// whose Gram entries are binary32 values).  The sums run over l (the sum
// index) with the rows i = lane + 32 s of every segment s advancing
// together; segments whose rows all exceed l are skipped (warp-uniform).
constexpr int kBuildTSegs = 4;  // 32-row segments: n <= 128
constexpr int kBuildTPad = 64;  // spare entries after each warp's triangle (no read ever reaches them)
constexpr int kBuildTStage = 8;  // rows of a slot whose loads are issued together

// SEGS >= ceil(n / 32) 32-row segments (2, 3 or kBuildTSegs): the staging
// and the accumulators are sized for this n, which keeps the registers, and
// so the warps resident per SM, in line with the work (n = 64: two segments).
template <class F, int SEGS>
__global__ void k_build_t(double* __restrict__ Tst, int64_t p, int n) {
  extern __shared__ __align__(16) unsigned char tsm_raw[];
  F* tsm = reinterpret_cast<F*>(tsm_raw);
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int np = n * (n + 1) / 2;
  F* t = tsm + static_cast<size_t>(wl) * (np + kBuildTPad);
  const int64_t blk = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + wl;
  if (blk >= p) return;  // warp-level work only: no CTA barrier below
  double* g = Tst + blk * n * n;
  // stage the upper triangle kBuildTStage rows at a time: all their loads are
  // in flight before the first store (one DRAM round trip per row otherwise)
  for (int i0 = 0; i0 < n; i0 += kBuildTStage) {
    double v[kBuildTStage][SEGS];
#pragma unroll
    for (int r = 0; r < kBuildTStage; ++r)
#pragma unroll
      for (int s = 0; s < SEGS; ++s) {
        const int i = i0 + r, c = i + lane + 32 * s;
        v[r][s] = (i < n && c < n) ? g[i * n + c] : 0.0;
      }
#pragma unroll
    for (int r = 0; r < kBuildTStage; ++r)
#pragma unroll
      for (int s = 0; s < SEGS; ++s) {
        const int i = i0 + r, c = i + lane + 32 * s;
        if (i < n && c < n) t[c * (c + 1) / 2 + i] = static_cast<F>(v[r][s]);
      }
  }
  __syncwarp();
  // columns j0 .. j0+3 per pass: T(i,j) = -tau_j sum_{l=i}^{j-1} T(i,l) G(l,j).
  // The sum over the finished columns l < j0 is shared by the four (one
  // load of T(i,l) feeds four FMAs, G(l, j0..j0+3) are broadcast); the terms
  // l in [j0, j) follow in registers, column by column; the four columns of
  // T are then written over theirs of G (read only in this pass).
  for (int j0 = 0; j0 < n; j0 += 4) {
    const int nj = n - j0 < 4 ? n - j0 : 4;
    const F* gc[4];
  #pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int j = j0 + (jj < nj ? jj : 0);
      gc[jj] = t + j * (j + 1) / 2;  // column j: G(l, j) for l < j, tau_j at l = j
    }
    F acc[4][SEGS];
  #pragma unroll
    for (int jj = 0; jj < 4; ++jj)
  #pragma unroll
      for (int s = 0; s < SEGS; ++s) acc[jj][s] = F(0);
    const F* tl = t;  // column l of T, advanced by l + 1 entries per step
    for (int l = 0; l < j0; l += 4) {  // j0 is a multiple of 4: whole groups
      const F* t1 = tl + l + 1;
      const F* t2 = t1 + l + 2;
      const F* t3 = t2 + l + 3;
      F gv[4][4];
  #pragma unroll
      for (int jj = 0; jj < 4; ++jj)
  #pragma unroll
        for (int u = 0; u < 4; ++u) gv[jj][u] = gc[jj][l + u];
  #pragma unroll
      for (int s = 0; s < SEGS; ++s) {
        if (32 * s > l + 3) break;  // rows of this and later segments all exceed l + 3
        const int i = lane + 32 * s;
        F x0 = F(0), x1 = F(0), x2 = F(0), x3 = F(0);  // rows below a column's diagonal add 0
        if (i <= l) x0 = tl[i];
        if (i <= l + 1) x1 = t1[i];
        if (i <= l + 2) x2 = t2[i];
        if (i <= l + 3) x3 = t3[i];
  #pragma unroll
        for (int jj = 0; jj < 4; ++jj)
          acc[jj][s] = fma(x3, gv[jj][3], fma(x2, gv[jj][2], fma(x1, gv[jj][1], fma(x0, gv[jj][0], acc[jj][s]))));
      }
      tl = t3 + l + 4;
    }
    // the block's own columns in order: T(i, j) gains the terms l in [j0, j)
    F tv[4][SEGS];
  #pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      if (jj < nj) {  // warp-uniform
        const int j = j0 + jj;
        const F tj = gc[jj][j];
  #pragma unroll
        for (int s = 0; s < SEGS; ++s) {
          const int i = lane + 32 * s;
          F a = acc[jj][s];
  #pragma unroll
          for (int ll = 0; ll < jj; ++ll) a = fma(tv[ll][s], gc[jj][j0 + ll], a);
          tv[jj][s] = i < j ? -tj * a : (i == j ? tj : F(0));
        }
      }
    }
    __syncwarp();  // every lane has read the block's columns of G
  #pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      if (jj < nj) {
        const int j = j0 + jj;
        F* tcol = t + j * (j + 1) / 2;
  #pragma unroll
        for (int s = 0; s < SEGS; ++s) {
          const int i = lane + 32 * s;
          if (i < j) tcol[i] = tv[jj][s];
        }
      }
    }
    __syncwarp();
  }
  for (int i = 0; i < n; ++i)
    for (int c = i + lane; c < n; c += 32) g[i * n + c] = static_cast<double>(t[c * (c + 1) / 2 + i]);
}

// Few slots (the upper tree levels): one slot per CTA, column c of T formed
// by thread c with no barrier in between.  The column recursion's T has the
// inverse diag(1/tau) + (the strict upper triangle of G) -- exactly, for the
// computed tau and G (by induction: T_j = [T, a; 0, tau_j] with a = -tau_j T
// G(0:j, j) has the inverse [T^-1, G(0:j, j); 0, 1/tau_j]) -- so each column
// is an independent back substitution: T(c,c) = tau_c and, for i = c-1 down
// to 0, T(i,c) = -tau_i sum_{k=i+1}^{c} G(i,k) T(k,c) (tau_i = 0 gives a zero
// row, as the recursion does).  The sum runs over k ascending in two
// interleaved chains.  G and T in shared memory, n x n each.
template <class F>
__global__ void __launch_bounds__(128) k_build_t_cta(double* __restrict__ Tst, int n) {
  extern __shared__ __align__(16) unsigned char tsm_raw[];
  F* G = reinterpret_cast<F*>(tsm_raw);  // n x n: tau on the diagonal, G above it
  F* T = G + n * n;                       // n x n: column c is thread c's
  double* g = Tst + static_cast<int64_t>(blockIdx.x) * n * n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, c = idx - i * n;
    G[idx] = c >= i ? static_cast<F>(g[idx]) : F(0);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    T[c * n + c] = G[c * n + c];
    for (int i = c - 1; i >= 0; --i) {
      F a0 = F(0), a1 = F(0);
      int k = i + 1;
      for (; k + 1 <= c; k += 2) {
        a0 = fma(G[i * n + k], T[k * n + c], a0);
        a1 = fma(G[i * n + k + 1], T[(k + 1) * n + c], a1);
      }
      if (k <= c) a0 = fma(G[i * n + k], T[k * n + c], a0);
      T[i * n + c] = -G[i * n + i] * (a0 + a1);
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int i = idx / n, c = idx - i * n;
    if (c >= i) g[idx] = static_cast<double>(T[idx]);
  }
}

template <class F>
static cudaError_t build_t_typed(double* Tst, int64_t p, int n, int sms, cudaStream_t st) {
  const size_t np = static_cast<size_t>(n) * (n + 1) / 2;
  if (p < 2 * static_cast<int64_t>(sms)) {
    // few slots: latency decides, so one CTA per slot, a thread per column
    const size_t smem = 2 * static_cast<size_t>(n) * n * sizeof(F);
    cudaError_t e = cudaFuncSetAttribute(k_build_t_cta<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_build_t_cta<F><<<static_cast<unsigned>(p), 128, smem, st>>>(Tst, n);
    return cudaGetLastError();
  }
  // many slots: one warp per slot, as many warps (<= 16) as packed triangles fit in 220 KB
  const size_t per_warp = (np + kBuildTPad) * sizeof(F);
  int warps = static_cast<int>((220u * 1024u) / per_warp);
  warps = warps < 1 ? 1 : (warps > 16 ? 16 : warps);
  const size_t smem = static_cast<size_t>(warps) * per_warp;
  const int64_t grid = (p + warps - 1) / warps;
  // (the column-by-column form took n <= 32 with four segments' registers, to
  // leave room for the tree's CTA beside it; the four-column form with one
  // segment is faster there too: 8,000,000 x 25 FP64 Step 2 4.11 -> 3.94 ms)
  const int segs = (n + 31) / 32;
  auto fn = segs == 1 ? k_build_t<F, 1> : segs == 2 ? k_build_t<F, 2> : segs == 3 ? k_build_t<F, 3> : k_build_t<F, 4>;
  if (segs > kBuildTSegs) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fn<<<static_cast<unsigned>(grid), 32 * warps, smem, st>>>(Tst, p, n);
  return cudaGetLastError();
}

cudaError_t launch_build_t(double* Tst, int64_t p, int n, bool binary32, cudaStream_t st) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return binary32 ? build_t_typed<float>(Tst, p, n, sms, st) : build_t_typed<double>(Tst, p, n, sms, st);
}

// G = sum over the nparts partials, in index order (one thread per entry).
__global__ void k_gram_reduce(const double* __restrict__ part, int nparts, int n, double* __restrict__ G,
                              int32_t* status) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  double s = 0.0;
  for (int p = 0; p < nparts; ++p) s += part[static_cast<int64_t>(p) * n * n + e];
  if (!isfinite(s)) set_status(status, TSQR_ERR_NONFINITE);
  G[e] = s;
}

cudaError_t launch_gram_reduce(const double* part, int nparts, int n, double* G, int32_t* status,
                               cudaStream_t st) {
  const int threads = 256;
  k_gram_reduce<<<(n * n + threads - 1) / threads, threads, 0, st>>>(part, nparts, n, G, status);
  return cudaGetLastError();
}

}  // namespace tsqr
