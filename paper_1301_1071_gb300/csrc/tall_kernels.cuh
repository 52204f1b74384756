// tall_kernels.cuh -- the tall passes of the comparators and of the adjoint.
//
//   k_gram   : partial Grams X^T Y over row chunks (binary64 accumulation),
//              one n x n partial per CTA; k_gram_reduce sums the partials in
//              a fixed order (deterministic, no atomics).  A^T A is the
//              Cholesky-QR reduction of Sec. II-A (Alg. 1); dQ^T Q feeds the
//              adjoint.
//   k_rowmul : out_r = X_r M1 + Y_r M2 for every row r (M1, M2 n x n,
//              binary64, converted to the compute type).  Q = A R^{-1}
//              (Sec. II-C) and dA = dQ R^{-T} + Q (C R^{-T}) of the adjoint.
#pragma once

#include "device.cuh"
#include "layout.cuh"

namespace tsqr {

// Each thread accumulates a TG x TG tile of X^T Y in type A (binary64, or
// binary32 for the adjoint of binary32 data: the per-CTA partial Grams are
// then summed in binary64); TG (4 or 5) is chosen per n to waste the fewest
// padded products (n = 25: 5, n = 64: 4).
// X, Y: m x n (storage S).  Rows are processed in chunks of `chunk` rows,
// chunks dealt to CTAs round-robin.  part: gridDim.x blocks of n x n binary64.
// Y == X is allowed (symmetric use).  Dynamic smem: 2 * chunk * n * sizeof(S) + 16.
template <class S, int TG, class A>
__global__ void k_gram(const S* __restrict__ X, const S* __restrict__ Y, int64_t m, int n, int chunk,
                       double* __restrict__ part, int32_t* status) {
  extern __shared__ __align__(128) unsigned char smem[];
  S* sx = reinterpret_cast<S*>(smem);
  S* sy = reinterpret_cast<S*>(smem + align_up((size_t)chunk * n * sizeof(S), 16));
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * align_up((size_t)chunk * n * sizeof(S), 16));
  const bool same = (X == Y);
  const int nt = (n + TG - 1) / TG;
  const int ntiles = nt * nt;
  const int NG = blockDim.x / ntiles > 0 ? blockDim.x / ntiles : 1;  // row groups
  const int tile = threadIdx.x % ntiles, g = threadIdx.x / ntiles;
  const bool active = threadIdx.x < ntiles * NG;
  const int k0 = (tile / nt) * TG, l0 = (tile % nt) * TG;
  A acc[TG][TG];
#pragma unroll
  for (int i = 0; i < TG; ++i)
#pragma unroll
    for (int j = 0; j < TG; ++j) acc[i][j] = A(0);

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int64_t nchunks = (m + chunk - 1) / chunk;
  uint32_t parity = 0;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int64_t r0 = c * chunk;
    const int rows = static_cast<int>(m - r0 < chunk ? m - r0 : chunk);
    if (!cta_load_bulk(sx, X + r0 * n, static_cast<int64_t>(rows) * n, bar, parity, status)) return;
    if (!same)
      if (!cta_load_bulk(sy, Y + r0 * n, static_cast<int64_t>(rows) * n, bar, parity, status)) return;
    __syncthreads();
    const S* ys = same ? sx : sy;
    if (active) {
      for (int r = g; r < rows; r += NG) {
        A xv[TG], yv[TG];
#pragma unroll
        for (int i = 0; i < TG; ++i) {
          xv[i] = (k0 + i < n) ? static_cast<A>(sx[r * n + k0 + i]) : A(0);
          yv[i] = (l0 + i < n) ? static_cast<A>(ys[r * n + l0 + i]) : A(0);
        }
#pragma unroll
        for (int i = 0; i < TG; ++i)
#pragma unroll
          for (int j = 0; j < TG; ++j) acc[i][j] = fma(xv[i], yv[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  // reduce the NG row groups through shared memory (reuse the stage)
  double* red = reinterpret_cast<double*>(smem);
  const size_t need = (size_t)NG * n * n * sizeof(double);
  const size_t have = 2 * align_up((size_t)chunk * n * sizeof(S), 16);
  double* P = part + static_cast<int64_t>(blockIdx.x) * n * n;
  if (need <= have) {
    if (active) {
#pragma unroll
      for (int i = 0; i < TG; ++i)
#pragma unroll
        for (int j = 0; j < TG; ++j)
          if (k0 + i < n && l0 + j < n) red[(size_t)g * n * n + (k0 + i) * n + (l0 + j)] = acc[i][j];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      double s = 0.0;
      for (int gg = 0; gg < NG; ++gg) s += red[(size_t)gg * n * n + e];
      P[e] = s;
    }
  } else {
    // sequential accumulation in global memory, group by group (deterministic)
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) P[e] = 0.0;
    __syncthreads();
    for (int gg = 0; gg < NG; ++gg) {
      if (active && g == gg) {
#pragma unroll
        for (int i = 0; i < TG; ++i)
#pragma unroll
          for (int j = 0; j < TG; ++j)
            if (k0 + i < n && l0 + j < n) P[(k0 + i) * n + (l0 + j)] += acc[i][j];
      }
      __syncthreads();
    }
  }
}

// out_r = X_r M1 + Y_r M2 (X or Y may be NULL).  Same thread tiling as
// k_form_q: R rows x NPC columns per thread, CS column slices, NRG row groups.
// The stage holds `srows` rows; rows per CTA b <= srows (one input) or
// b <= srows/2 (both X and Y: two halves).
template <class S, class T, int NPC, int R, int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
    k_rowmul(const S* X, const double* __restrict__ M1, const S* Yin, const double* __restrict__ M2, int64_t m,
             int n, int b, int srows, int CS, int NRG, int skew, S* out, int32_t* status) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int NT = blockDim.x;
  const int B = 32 * NRG * R;
  const int NPAD = NPC * CS;
  const RowMulSmem L(srows, n, NPAD, sizeof(S), sizeof(T));
  (void)B;
  S* sx = reinterpret_cast<S*>(smem + L.sx);
  S* sy = sx + static_cast<size_t>(b) * n;  // second half (only when both inputs)
  T* m1 = reinterpret_cast<T*>(smem + L.m1);
  T* m2 = reinterpret_cast<T*>(smem + L.m2);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cs = warp % CS, rg = warp / CS;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * b;
  const int rows = static_cast<int>(m - row0 < b ? m - row0 : b);
  const int rbase = rg * 32 * R + lane;  // thread rows rbase + 32 q, as in k_local_qr
  (void)NRG;

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  for (int idx = tid; idx < n * NPAD; idx += NT) {
    const int k = idx / NPAD, c = idx % NPAD;
    m1[idx] = (X && c < n) ? static_cast<T>(M1[k * n + c]) : T(0);
    m2[idx] = (Yin && c < n) ? static_cast<T>(M2[k * n + c]) : T(0);
  }
  __syncthreads();
  uint32_t parity = 0;
  if (X) {
    if (!cta_load_bulk(sx, X + row0 * n, static_cast<int64_t>(rows) * n, bar, parity, status)) return;
  }
  if (Yin) {
    S* dst = X ? sy : sx;
    if (!cta_load_bulk(dst, Yin + row0 * n, static_cast<int64_t>(rows) * n, bar, parity, status)) return;
  }
  __syncthreads();
  const S* ys = X ? sy : sx;

  T acc[R][NPC];
#pragma unroll
  for (int q = 0; q < R; ++q)
#pragma unroll
    for (int c = 0; c < NPC; ++c) acc[q][c] = T(0);
  // skew != 0: lane l takes the columns in the cyclic order starting at
  // l mod n (bank-conflict-free reads of one column of consecutive rows)
  int k = skew ? lane % n : 0;
  for (int step = 0; step < n; ++step, k = (k + 1 == n) ? 0 : k + 1) {
    if (X) {
      T w[NPC];
#pragma unroll
      for (int c = 0; c < NPC; ++c) w[c] = m1[k * NPAD + cs + c * CS];
      const S* xp = sx + rbase * n + k;  // advanced by 32 rows per step
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int r = rbase + 32 * q;
        const T xv = (r < rows) ? static_cast<T>(*xp) : T(0);
        xp += 32 * n;
#pragma unroll
        for (int c = 0; c < NPC; ++c) acc[q][c] = fma(xv, w[c], acc[q][c]);
      }
    }
    if (Yin) {
      T w[NPC];
#pragma unroll
      for (int c = 0; c < NPC; ++c) w[c] = m2[k * NPAD + cs + c * CS];
      const S* yp = ys + rbase * n + k;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int r = rbase + 32 * q;
        const T yv = (r < rows) ? static_cast<T>(*yp) : T(0);
        yp += 32 * n;
#pragma unroll
        for (int c = 0; c < NPC; ++c) acc[q][c] = fma(yv, w[c], acc[q][c]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int r = rbase + 32 * q;
    if (r < rows) {
#pragma unroll
      for (int c = 0; c < NPC; ++c) {
        const int k = cs + c * CS;
        if (k < n) sx[r * n + k] = static_cast<S>(acc[q][c]);
      }
    }
  }
  fence_proxy_async_smem();
  __syncthreads();
  cta_store_bulk(out + row0 * n, sx, static_cast<int64_t>(rows) * n);
}

}  // namespace tsqr
