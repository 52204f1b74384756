// qr_kernels.cuh -- the two kernels of direct TSQR (Sec. III-B):
//
//   k_local_qr : Step 1 (and every level of the recursive Step 2, Alg. 2).
//                One CTA per row block A_i (b x n).  The block is staged into
//                shared memory with bulk TMA, then held in REGISTERS: each
//                thread owns R rows x NPC columns (columns dealt cyclically
//                over CS column slices, one slice per warp).  Householder QR
//                column by column; one CTA-wide reduction per column computes
//                x^T A over the active rows, which yields at once ||x||^2, the
//                dots with the trailing columns and the Gram entries v_i^T v_j
//                needed for the compact-WY T factor.  Outputs Y_i (unit lower
//                trapezoid, written over the block), R_i and T_i (binary64).
//
//   k_form_q   : Step 3.  Q_i = Q1_i Q2_i = [C_i; 0] - Y_i (T_i (Y_top_i^T C_i))
//                with C_i = Q2_i (n x n); fused epilogue with bulk stores.
//
// Householder convention: alpha = x_1, sigma = ||x||, beta = -copysign(sigma,
// alpha), v = (x - beta e_1)/(alpha - beta), tau = (beta - alpha)/beta,
// H = I - tau v v^T; a zero column gives tau = 0 (H = I).
#pragma once

#include <type_traits>

#include "device.cuh"
#include "df64.cuh"
#include "layout.cuh"

namespace tsqr {

// ---------------------------------------------------------------------------
// Arithmetic traits: storage type S, compute type T.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double dev_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dev_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double dev_copysign(double a, double b) { return copysign(a, b); }
__device__ __forceinline__ float dev_copysign(float a, float b) { return copysignf(a, b); }

// ---------------------------------------------------------------------------
// Step 1: local Householder QR of one row block per CTA.
//   A    : m x n row-major (storage S); block i = rows [i*b, min(i*b+b, m)).
//   Y    : output, same shape; may alias A (the block is staged first).  NULL
//          = R-only mode (no Y, no T).
//   Rst  : p blocks of n x n binary64 (R_i, upper triangular, raw signs).
//   Tst  : p blocks of n x n binary64 (T_i, upper triangular), or NULL.
// Launch: blockDim = 32*CS*NRG <= MAXT, gridDim = p, dynamic smem = LocalQrSmem.
// ---------------------------------------------------------------------------
template <class S, class T, int NPC, int R, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_local_qr(const S* __restrict__ A, int64_t m, int n, int b, int CS, int NRG,
                           S* Y, double* __restrict__ Rst, double* __restrict__ Tst,
                           int32_t* status) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int NT = blockDim.x;
  const int NW = NT >> 5;
  const int B = 32 * NRG * R;
  const int NPAD = NPC * CS;
  const LocalQrSmem L(B, n, NW, NPAD, sizeof(S), sizeof(T));
  S* stage = reinterpret_cast<S*>(smem + L.stage);
  T* gram = reinterpret_cast<T*>(smem + L.stage);  // reused during the loop
  T* red = reinterpret_cast<T*>(smem + L.red);
  // pivot column, double-buffered by the parity of j: in phase C the warps
  // owning column j+1 publish it while other column slices still read x_j
  T* xbuf = reinterpret_cast<T*>(smem + L.xcol);
  T* piv = reinterpret_cast<T*>(smem + L.piv);
  T* ssum = reinterpret_cast<T*>(smem + L.ssum);
  T* dk = reinterpret_cast<T*>(smem + L.dk);
  T* taus = reinterpret_cast<T*>(smem + L.tau);
  T* sc = reinterpret_cast<T*>(smem + L.scal);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cs = warp % CS, rg = warp / CS;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * b;
  const int rows = static_cast<int>(m - row0 < b ? m - row0 : b);
  const int RS = 32 * NRG;  // row stride between a thread's rows

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  for (int k = tid; k < NPAD; k += NT) dk[k] = T(0);
  __syncthreads();
  uint32_t parity = 0;
  if (!cta_load_bulk(stage, A + row0 * n, static_cast<int64_t>(rows) * n, bar, parity, status)) return;
  __syncthreads();

  T a[R][NPC];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int r = rg * 32 + lane + q * RS;
#pragma unroll
    for (int c = 0; c < NPC; ++c) {
      const int k = cs + c * CS;
      a[q][c] = (r < rows && k < n) ? static_cast<T>(stage[r * n + k]) : T(0);
    }
  }
  // Double-float compute: scale the block by a power of two (exact) so that
  // its largest entry is ~1 and products of small entries stay in binary32
  // range.  Y and T are invariant under the scaling; R is unscaled on output.
  int scale_exp = 0;
  if constexpr (std::is_same<T, df64>::value) {
    float mx = 0.0f;
#pragma unroll
    for (int q = 0; q < R; ++q)
#pragma unroll
      for (int c = 0; c < NPC; ++c) mx = fmaxf(mx, fabsf(a[q][c].hi));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    float* wmax = reinterpret_cast<float*>(red);
    if (lane == 0) wmax[warp] = mx;
    __syncthreads();
    float bm = 0.0f;
    for (int w = 0; w < NW; ++w) bm = fmaxf(bm, wmax[w]);
    if (bm > 0.0f && isfinite(bm)) {
      int e;
      frexpf(bm, &e);
      scale_exp = e;  // bm = f * 2^e, f in [0.5, 1)
#pragma unroll
      for (int q = 0; q < R; ++q)
#pragma unroll
        for (int c = 0; c < NPC; ++c) a[q][c] = scale2(a[q][c], -scale_exp);
    }
  }
  __syncthreads();  // stage is reused for the Gram matrix from here on

  // publish pivot column 0 and pivot row 0
  if (cs == 0) {
#pragma unroll
    for (int q = 0; q < R; ++q) xbuf[rg * 32 + lane + q * RS] = a[q][0];
  }
  if (rg == 0 && lane == 0) {
#pragma unroll
    for (int c = 0; c < NPC; ++c) piv[cs + c * CS] = a[0][c];
  }
  __syncthreads();

  for (int j = 0; j < n; ++j) {
    const T* xcol = xbuf + (j & 1) * B;   // x_j
    T* xnext = xbuf + ((j + 1) & 1) * B;  // x_{j+1}
    // ---- phase A: s = x^T A over the thread's active rows, CTA reduction
    T s[NPC];
#pragma unroll
    for (int c = 0; c < NPC; ++c) s[c] = T(0);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int r = rg * 32 + lane + q * RS;
      const T xq = (r >= j) ? xcol[r] : T(0);
#pragma unroll
      for (int c = 0; c < NPC; ++c) s[c] = fma(xq, a[q][c], s[c]);
    }
    TransposeReduce<NPC, 16>::run(s, lane, 0, NPC, red + warp * 32);
    __syncthreads();

    // ---- phase B: warp 0 combines, forms the reflector and the update coefficients
    if (warp == 0) {
      for (int k = lane; k < n; k += 32) {
        const int kcs = k % CS, kc = k / CS;
        T acc = T(0);
        for (int g = 0; g < NRG; ++g) acc += red[(g * CS + kcs) * 32 + kc];
        ssum[k] = acc;
      }
      __syncwarp();
      if (lane == 0) {
        const T alpha = piv[j];
        const T sigma = dev_sqrt(ssum[j]);
        T beta, amb, scal, ib, tau;
        if (sigma == T(0)) {
          beta = alpha; amb = T(0); scal = T(0); ib = T(0); tau = T(0);
        } else {
          beta = -dev_copysign(sigma, alpha);
          amb = alpha - beta;
          scal = T(1) / amb;
          ib = T(1) / beta;
          tau = (beta - alpha) * ib;
        }
        sc[0] = beta; sc[1] = amb; sc[2] = scal; sc[3] = ib;
        sc[4] = (sigma == T(0)) ? T(1) : T(0);  // identity reflector
        taus[j] = tau;
      }
      __syncwarp();
      const T beta = sc[0], scal = sc[2], ib = sc[3];
      for (int k = lane; k < NPAD; k += 32) {
        if (k > j && k < n) {
          dk[k] = (piv[k] - ssum[k] * ib) * scal;
        } else if (k < j) {
          gram[k * n + j] = scal * (ssum[k] - beta * piv[k]);
        }
      }
    }
    __syncthreads();

    // ---- phase C: trailing update, store v_j, pivot row = R row j,
    //      publish pivot column/row j+1
    {
      const T beta = sc[0], scal = sc[2], ib = sc[3];
      const bool ident = sc[4] != T(0);
      // first local column index with global column > j (warp-uniform)
      const int c0 = (j >= cs) ? (j - cs) / CS + 1 : 0;
      const bool own_j = (cs == j % CS);
      const int cj = j / CS;
      T d[NPC];
#pragma unroll
      for (int c = 0; c < NPC; ++c) d[c] = (c >= c0) ? dk[cs + c * CS] : T(0);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int r = rg * 32 + lane + q * RS;
        if (r >= j) {
          const T xq = xcol[r];
          if (r > j) {
#pragma unroll
            for (int c = 0; c < NPC; ++c)
              if (c >= c0) a[q][c] = fma(-d[c], xq, a[q][c]);
            if (own_j) {
#pragma unroll
              for (int c = 0; c < NPC; ++c)
                if (c == cj) a[q][c] = xq * scal;
            }
          } else if (!ident) {  // pivot row: R_jj = beta, R_jk = (x^T a_k) / beta
#pragma unroll
            for (int c = 0; c < NPC; ++c) {
              if (c >= c0 && cs + c * CS < n) a[q][c] = ssum[cs + c * CS] * ib;
              if (own_j && c == cj) a[q][c] = beta;
            }
          }
        }
      }
      if (j + 1 < n) {
        const int jn = j + 1;
        if (cs == jn % CS) {
          const int cn = jn / CS;
#pragma unroll
          for (int c = 0; c < NPC; ++c) {
            if (c == cn) {
#pragma unroll
              for (int q = 0; q < R; ++q) xnext[rg * 32 + lane + q * RS] = a[q][c];
            }
          }
        }
        const int qp = jn / RS, wp = jn % RS;
        if (rg == wp / 32 && lane == wp % 32) {
#pragma unroll
          for (int q = 0; q < R; ++q) {
            if (q == qp) {
#pragma unroll
              for (int c = 0; c < NPC; ++c) piv[cs + c * CS] = a[q][c];
            }
          }
        }
      }
    }
    __syncthreads();
  }

  // ---- R_i (raw signs) for rows < n
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int r = rg * 32 + lane + q * RS;
    if (r < n) {
#pragma unroll
      for (int c = 0; c < NPC; ++c) {
        const int k = cs + c * CS;
        if (k < n)
          Rst[static_cast<int64_t>(blockIdx.x) * n * n + r * n + k] =
              (k >= r && r < rows) ? ldexp(static_cast<double>(a[q][c]), scale_exp) : 0.0;
      }
    }
  }

  if (Y == nullptr) return;  // R-only mode (indirect TSQR)

  // ---- T_i from the Gram entries (in place, column by column), warp 0
  if (warp == 0) {
    for (int j = 0; j < n; ++j) {
      T tv[4];  // n <= 128 rows of T per column: 4 per lane
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int i = lane + 32 * t;
        T acc = T(0);
        if (i < j) {
          for (int l = i; l < j; ++l) {
            const T til = (l == i) ? taus[i] : gram[i * n + l];
            acc = fma(til, gram[l * n + j], acc);
          }
        }
        tv[t] = -taus[j] * acc;
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int i = lane + 32 * t;
        if (i < j) gram[i * n + j] = tv[t];
      }
      __syncwarp();
    }
    double* Tout = Tst + static_cast<int64_t>(blockIdx.x) * n * n;
    for (int idx = lane; idx < n * n; idx += 32) {
      const int i = idx / n, k = idx % n;
      Tout[idx] = (k > i) ? static_cast<double>(gram[idx]) : (k == i ? static_cast<double>(taus[i]) : 0.0);
    }
  }
  __syncthreads();

  // ---- Y_i back through shared memory, bulk store
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int r = rg * 32 + lane + q * RS;
    if (r < rows) {
#pragma unroll
      for (int c = 0; c < NPC; ++c) {
        const int k = cs + c * CS;
        if (k < n) stage[r * n + k] = static_cast<S>(a[q][c]);
      }
    }
  }
  fence_proxy_async_smem();
  __syncthreads();
  cta_store_bulk(Y + row0 * n, stage, static_cast<int64_t>(rows) * n);
}

// ---------------------------------------------------------------------------
// Step 3: Q_i = [C_i; 0] - Y_i W_i, W_i = T_i (Y_top_i^T C_i).
//   Yg  : m x n (storage S), Y_i per block as written by k_local_qr.
//   Tg  : p blocks of n x n binary64.  Cg: p blocks of n x n binary64 (Q2_i).
//   Qg  : output m x n (storage S); may alias Yg.
// ---------------------------------------------------------------------------
template <class S, class T, int NPC, int R, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_form_q(const S* Yg, int64_t m, int n, int b, int srows, int CS, int NRG,
                                                     const double* __restrict__ Tg, const double* __restrict__ Cg,
                                                     int64_t cblocks, S* Qg, int32_t* status) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int NT = blockDim.x;
  const int NPAD = NPC * CS;
  const FormQSmem L(srows, n, NPAD, sizeof(S), sizeof(T));
  S* stage = reinterpret_cast<S*>(smem + L.stage);
  T* Wm = reinterpret_cast<T*>(smem + L.wm);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cs = warp % CS, rg = warp / CS;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * b;
  const int rows = static_cast<int>(m - row0 < b ? m - row0 : b);
  const int RS = 32 * NRG;
  const int ntop = rows < n ? rows : n;
  const S* Yb = Yg + row0 * n;

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  const int64_t cb = cblocks == 1 ? 0 : static_cast<int64_t>(blockIdx.x);
  const double* Tb = Tg + static_cast<int64_t>(blockIdx.x) * n * n;
  const double* Cb = Cg + cb * n * n;

  // X = Y_top^T C  (Y_top unit lower triangular, rows < ntop, read from
  // global memory before any row of this block is overwritten), into Wm
  for (int idx = tid; idx < n * NPAD; idx += NT) {
    const int k = idx / NPAD, c = idx % NPAD;
    T acc = T(0);
    if (c < n && k < ntop) {
      acc = static_cast<T>(Cb[k * n + c]);
      for (int r = k + 1; r < ntop; ++r)
        acc = fma(static_cast<T>(Yb[r * n + k]), static_cast<T>(Cb[r * n + c]), acc);
    }
    Wm[idx] = acc;
  }
  __syncthreads();
  // W = T X in place, one thread per column: row k of W only needs rows >= k of X
  for (int c = tid; c < n; c += NT) {
    for (int k = 0; k < n; ++k) {
      T acc = T(0);
      for (int i = k; i < n; ++i) acc = fma(static_cast<T>(Tb[k * n + i]), Wm[i * NPAD + c], acc);
      Wm[k * NPAD + c] = acc;
    }
  }
  __syncthreads();

  // Q rows = [C; 0] - Y W, chunk by chunk of `srows` staged rows
  uint32_t parity = 0;
  for (int c0 = 0; c0 < rows; c0 += srows) {
    const int crows = rows - c0 < srows ? rows - c0 : srows;
    if (!cta_load_bulk(stage, Yb + static_cast<int64_t>(c0) * n, static_cast<int64_t>(crows) * n, bar, parity,
                       status))
      return;
    T acc[R][NPC];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int r = c0 + rg * 32 + lane + q * RS;  // row within the block
#pragma unroll
      for (int c = 0; c < NPC; ++c) {
        const int k = cs + c * CS;
        acc[q][c] = (r < ntop && k < n) ? static_cast<T>(Cb[r * n + k]) : T(0);
      }
    }
    for (int k = 0; k < n; ++k) {
      T w[NPC];
#pragma unroll
      for (int c = 0; c < NPC; ++c) w[c] = Wm[k * NPAD + cs + c * CS];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int rl = rg * 32 + lane + q * RS;  // row within the chunk
        const int r = c0 + rl;
        T y = T(0);
        if (rl < crows) y = (k < r) ? static_cast<T>(stage[rl * n + k]) : (k == r ? T(1) : T(0));
#pragma unroll
        for (int c = 0; c < NPC; ++c) acc[q][c] = fma(-y, w[c], acc[q][c]);
      }
    }
    __syncthreads();  // every read of this chunk in shared memory is done
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int rl = rg * 32 + lane + q * RS;
      if (rl < crows) {
#pragma unroll
        for (int c = 0; c < NPC; ++c) {
          const int k = cs + c * CS;
          if (k < n) stage[rl * n + k] = static_cast<S>(acc[q][c]);
        }
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    cta_store_bulk(Qg + row0 * n + static_cast<int64_t>(c0) * n, stage, static_cast<int64_t>(crows) * n);
    __syncthreads();  // the stage is free again (bulk store read it, tail stores done)
  }
}

}  // namespace tsqr
