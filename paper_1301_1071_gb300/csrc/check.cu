// check.cu -- tsqr_accuracy: the accuracy metrics of a computed factorisation
// (Sec. I-B: ||Q^T Q - I||_2 and ||A - QR||_2 / ||R||_2; also
// ||A - QR||_F / ||A||_F) accumulated on the device in compensated
// arithmetic, so that they stay meaningful at the 1e-15 level for tall
// matrices: a plain binary64 sum over m = 8e6 rows errs by ~sqrt(m) eps.
//
// Every product x y enters a double-double accumulator (s, c) through the
// error-free transformations of Ogita, Rump and Oishi ("Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005): p = x y and its exact error
// fma(x, y, -p) (TwoProduct), then s + p and its exact error (Knuth's
// TwoSum); the errors are summed into c.  The result s + c is as accurate as
// a sum in twice the working precision.
//
// Layout of the work: CTA c takes the row chunks c, c + G, c + 2G, ... of
// `ch` rows each, staged in shared memory; thread t owns the upper-triangle
// pairs (i <= j) t, t + NT, ... of the n x n Gram.  Per chunk each thread
// adds q_ri q_rj of every staged row to its pairs.  With A (and R): each
// residual entry e_rj = a_rj - sum_k q_rk r_kj is one Dot2 sum over k
// (written over the staged a_rj), its square is summed in plain binary64
// (the norms need a few digits only), and the Gram E^T E of the residual
// (for its 2-norm) in plain binary64 too.  Each CTA writes its partial sums;
// a second kernel combines them in CTA order (deterministic: no atomics).
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/tsqr.h"
#include "check.h"

namespace tsqr {

namespace {

constexpr int kChkThreads = 512;
constexpr int kChkMaxPairs = (TSQR_NMAX * (TSQR_NMAX + 1) / 2 + kChkThreads - 1) / kChkThreads;

struct Acc2 {
  double s, c;
};

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  const double z = s - a;
  e = (a - (s - z)) + (b - z);
}

__device__ __forceinline__ void acc_prod(Acc2& a, double x, double y) {
  const double p = x * y;
  const double ep = fma(x, y, -p);
  double s, es;
  two_sum(a.s, p, s, es);
  a.s = s;
  a.c += es + ep;
}

// (i, j), i <= j, of the p-th entry of the row-major upper triangle of n x n
__device__ __forceinline__ void pair_of(int p, int n, int& i, int& j) {
  i = 0;
  while (p >= n - i) {
    p -= n - i;
    ++i;
  }
  j = i + p;
}

template <class S>
__global__ void __launch_bounds__(kChkThreads, 1)
    k_accuracy(const S* __restrict__ Q, const S* __restrict__ A, const double* __restrict__ R, int64_t m, int n,
               int ch, double* __restrict__ part) {
  extern __shared__ double sm[];
  double* qs = sm;              // ch x n rows of Q
  double* as = qs + ch * n;     // ch x n rows of A, then of E = A - QR
  double* rs = as + ch * n;     // n x n R
  double* red = rs + n * n;     // 2 x NT per-thread norms for the ordered CTA sum
  const int tid = threadIdx.x;
  const int np = n * (n + 1) / 2;
  int pi[kChkMaxPairs], pj[kChkMaxPairs];
  Acc2 g[kChkMaxPairs];
  double e2[kChkMaxPairs];
#pragma unroll
  for (int k = 0; k < kChkMaxPairs; ++k) {
    const int p = tid + k * kChkThreads;
    if (p < np) pair_of(p, n, pi[k], pj[k]);
    else pi[k] = pj[k] = 0;
    g[k] = Acc2{0.0, 0.0};
    e2[k] = 0.0;
  }
  double ssE = 0.0, ssA = 0.0;
  if (A)
    for (int idx = tid; idx < n * n; idx += kChkThreads) rs[idx] = R[idx];
  for (int64_t c = blockIdx.x; c * ch < m; c += gridDim.x) {
    const int64_t r0 = c * ch;
    const int rows = static_cast<int>(m - r0 < ch ? m - r0 : ch);
    __syncthreads();  // the previous chunk's readers are done
    for (int idx = tid; idx < rows * n; idx += kChkThreads) {
      qs[idx] = static_cast<double>(Q[r0 * n + idx]);
      if (A) as[idx] = static_cast<double>(A[r0 * n + idx]);
    }
    __syncthreads();
    for (int r = 0; r < rows; ++r) {
      const double* q = qs + r * n;
#pragma unroll
      for (int k = 0; k < kChkMaxPairs; ++k)
        if (tid + k * kChkThreads < np) acc_prod(g[k], q[pi[k]], q[pj[k]]);
    }
    if (A) {
      for (int idx = tid; idx < rows * n; idx += kChkThreads) {
        const int r = idx / n, j = idx % n;
        const double a = as[idx];
        Acc2 t{a, 0.0};
        for (int k = 0; k < n; ++k) acc_prod(t, -qs[r * n + k], rs[k * n + j]);
        const double e = t.s + t.c;
        ssA += a * a;
        ssE += e * e;
        as[idx] = e;  // only this thread reads or writes entry idx in this phase
      }
      __syncthreads();
      for (int r = 0; r < rows; ++r) {
        const double* e = as + r * n;
#pragma unroll
        for (int k = 0; k < kChkMaxPairs; ++k)
          if (tid + k * kChkThreads < np) e2[k] += e[pi[k]] * e[pj[k]];
      }
    }
  }
  // partials of this CTA: (s, c) per pair, then E^T E per pair, then the two
  // squared norms (per-thread values summed in thread order by thread 0)
  const int64_t stride = 3 * static_cast<int64_t>(np) + 2;
  double* out = part + blockIdx.x * stride;
#pragma unroll
  for (int k = 0; k < kChkMaxPairs; ++k) {
    const int p = tid + k * kChkThreads;
    if (p < np) {
      out[2 * p] = g[k].s;
      out[2 * p + 1] = g[k].c;
      out[2 * np + p] = e2[k];
    }
  }
  __syncthreads();
  red[tid] = ssE;
  red[kChkThreads + tid] = ssA;
  __syncthreads();
  if (tid == 0) {
    double se = 0.0, sa = 0.0;
    for (int t = 0; t < kChkThreads; ++t) {
      se += red[t];
      sa += red[kChkThreads + t];
    }
    out[3 * np] = se;
    out[3 * np + 1] = sa;
  }
}

// Combines the G partials in CTA order.  out (3 n^2 + 2 binary64):
// hi and lo of Q^T Q - I (full symmetric), E^T E, ||E||_F^2, ||A||_F^2.
__global__ void __launch_bounds__(256) k_accuracy_reduce(const double* __restrict__ part, int G, int n,
                                                          double* __restrict__ out) {
  const int np = n * (n + 1) / 2;
  const int64_t stride = 3 * static_cast<int64_t>(np) + 2;
  const int nn = n * n;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    Acc2 t{0.0, 0.0};
    double e = 0.0;
    for (int c = 0; c < G; ++c) {
      const double* q = part + c * stride;
      double s, es;
      two_sum(t.s, q[2 * p], s, es);
      t.s = s;
      t.c += es + q[2 * p + 1];
      e += q[2 * np + p];
    }
    int i, j;
    pair_of(p, n, i, j);
    double hi = t.s, lo = t.c;
    if (i == j) hi -= 1.0;  // exact: hi is within a factor 2 of 1 for any useful Q
    out[i * n + j] = out[j * n + i] = hi;
    out[nn + i * n + j] = out[nn + j * n + i] = lo;
    out[2 * nn + i * n + j] = out[2 * nn + j * n + i] = e;
  }
  if (threadIdx.x == 0) {
    double se = 0.0, sa = 0.0;
    for (int c = 0; c < G; ++c) {
      se += part[c * stride + 3 * np];
      sa += part[c * stride + 3 * np + 1];
    }
    out[3 * nn] = se;
    out[3 * nn + 1] = sa;
  }
}

}  // namespace

AccuracyGeom accuracy_geom(int64_t m, int n) {
  AccuracyGeom g;
  int ch = static_cast<int>(kAccuracySmemRows / static_cast<int64_t>(n));
  ch = ch > 128 ? 128 : (ch < 1 ? 1 : ch);
  g.ch = ch;
  const int64_t chunks = (m + ch - 1) / ch;
  g.grid = static_cast<int>(chunks < kAccuracyMaxParts ? chunks : kAccuracyMaxParts);
  const int64_t np = static_cast<int64_t>(n) * (n + 1) / 2;
  g.part_bytes = static_cast<size_t>(g.grid) * static_cast<size_t>(3 * np + 2) * sizeof(double);
  g.smem = (2 * static_cast<size_t>(ch) * n + static_cast<size_t>(n) * n + 2 * kChkThreads) * sizeof(double);
  return g;
}

cudaError_t launch_accuracy(int esz, const void* Q, const void* A, const double* R, int64_t m, int n,
                            double* part, double* out, cudaStream_t st) {
  const AccuracyGeom g = accuracy_geom(m, n);
  if (esz == 8) {
    cudaError_t e = cudaFuncSetAttribute(k_accuracy<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(g.smem));
    if (e != cudaSuccess) return e;
    k_accuracy<double><<<g.grid, kChkThreads, g.smem, st>>>(static_cast<const double*>(Q),
                                                            static_cast<const double*>(A), R, m, n, g.ch, part);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_accuracy<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(g.smem));
    if (e != cudaSuccess) return e;
    k_accuracy<float><<<g.grid, kChkThreads, g.smem, st>>>(static_cast<const float*>(Q),
                                                           static_cast<const float*>(A), R, m, n, g.ch, part);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_accuracy_reduce<<<1, 256, 0, st>>>(part, g.grid, n, out);
  return cudaGetLastError();
}

}  // namespace tsqr
