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

// Storage <-> compute conversions.  Double-float compute converts binary64
// with integer operations (split_scaled / to_double) so that no binary64
// arithmetic is spent on data movement; `shift` scales by 2^-shift (exact).
template <class T, class S>
__device__ __forceinline__ T to_compute(S x, int shift) {
  if constexpr (std::is_same<T, df64>::value) {
    return split_scaled(x, shift);
  } else {
    (void)shift;
    return static_cast<T>(x);
  }
}
template <class S, class T>
__device__ __forceinline__ S to_storage(T v) {
  if constexpr (std::is_same<T, df64>::value) {
    return to_double(v);
  } else {
    return static_cast<S>(v);
  }
}
// Householder scalars of one column from S_j = ||x||^2 and alpha = x_1:
// beta = -copysign(sqrt(S_j), alpha), scal = 1/(alpha - beta), ib = 1/beta,
// tau = (beta - alpha)/beta; a zero column gives the identity (tau = 0).
template <class T>
struct Reflector {
  T beta, scal, ib, tau;
  bool ident;
};
// binary64 reciprocal by Newton's iteration y <- y + y (1 - x y) from a
// binary32 seed (2^-24 -> 2^-48 -> below one ulp after two steps); outside
// the binary32 range the IEEE division is used.  Four dependent FMAs instead
// of a full division sequence on the slow binary64 unit.
__device__ __forceinline__ double recip_of(double x) {
  const double ax = fabs(x);
  if (!(ax > 1e-36 && ax < 1e36)) return 1.0 / x;
  double y = static_cast<double>(1.0f / static_cast<float>(x));
  y = fma(fma(-x, y, 1.0), y, y);
  y = fma(fma(-x, y, 1.0), y, y);
  return y;
}
__device__ __forceinline__ float recip_of(float x) { return 1.0f / x; }
// double-float reciprocal and square root without binary64 arithmetic, from
// a correctly rounded binary32 estimate and an exactly formed residual (a
// TwoSum of its two leading parts plus the TwoProduct error terms), so that
// only the final rounding to the pair remains (~2^-49 relative).
__device__ __forceinline__ df64 recip_of(df64 x) {
  // 1/x = y0 / (1 - e), e = 1 - x y0 = 1 - (p + pe) - (q + qe), |e| <= 2^-22:
  // y0 (1 + e + e^2).  pe is as large as e itself, so e is summed with TwoSums.
  const float y0 = 1.0f / x.hi;
  const float p = x.hi * y0, pe = fmaf(x.hi, y0, -p);  // x.hi y0 = p + pe
  const float q = x.lo * y0, qe = fmaf(x.lo, y0, -q);  // x.lo y0 = q + qe
  const df64 d2 = two_sum(1.0f - p, -pe);              // 1 - p is exact
  const df64 d3 = two_sum(d2.hi, -q);
  const df64 e = fast_two_sum(d3.hi, (d2.lo + d3.lo) - qe);
  const float r = y0 * e.hi, re = fmaf(y0, e.hi, -r);
  const float small = fmaf(y0, fmaf(e.hi, e.hi, e.lo), re);
  df64 y = fast_two_sum(y0, r);
  y.lo += small;
  return fast_two_sum(y.hi, y.lo);
}
__device__ __forceinline__ double sqrt_of(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_of(float x) { return sqrtf(x); }
__device__ __forceinline__ df64 sqrt_of(df64 x) {
  // s0 = sqrt(x.hi); r = x - s0^2 = (x.hi - p) - pe + x.lo summed with TwoSums;
  // sqrt(x) = s0 + c - c^2/(2 s0), c = r / (2 s0) carried as two words
  const float s0 = sqrtf(x.hi);
  if (s0 == 0.0f) return df64(0.0f, 0.0f);
  const float p = s0 * s0, pe = fmaf(s0, s0, -p);
  const df64 d2 = two_sum(x.hi - p, -pe);  // x.hi - p is exact
  const df64 d3 = two_sum(d2.hi, x.lo);
  const float rl = d2.lo + d3.lo;
  const float t = 2.0f * s0, h = 0.5f / s0;
  const float c0 = d3.hi * h;
  const float c1 = fmaf(fmaf(-c0, t, d3.hi) + rl, h, c0);      // r / (2 s0), rounded
  const float res = fmaf(-c1, t, d3.hi) + rl;                    // r - c1 (2 s0)
  const float clo = fmaf(res, h, (-c1 * c1) * h);                // the rest of c - c^2/(2 s0)
  df64 y = fast_two_sum(s0, c1);
  y.lo += clo;
  return fast_two_sum(y.hi, y.lo);
}
template <class T>
__device__ __forceinline__ Reflector<T> make_reflector(T Sj, T alpha) {
  Reflector<T> f;
  const T sigma = sqrt_of(Sj);
  if (sigma == T(0)) {
    f.beta = alpha; f.scal = T(0); f.ib = T(0); f.tau = T(0); f.ident = true;
  } else {
    f.beta = -dev_copysign(sigma, alpha);
    f.scal = recip_of(alpha - f.beta);
    f.ib = recip_of(f.beta);
    f.tau = (f.beta - alpha) * f.ib;
    f.ident = false;
  }
  return f;
}
template <class T>
__device__ __forceinline__ T shfl_from(T v, int src) {
  if constexpr (std::is_same<T, df64>::value) {
    return df64(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
  } else {
    return __shfl_sync(0xffffffffu, v, src);
  }
}
template <class T>
__device__ __forceinline__ T shfl_bcast(T v) {
  if constexpr (std::is_same<T, df64>::value) {
    return df64(__shfl_sync(0xffffffffu, v.hi, 0), __shfl_sync(0xffffffffu, v.lo, 0));
  } else {
    return __shfl_sync(0xffffffffu, v, 0);
  }
}

// Sum over the warp (every lane gets it).
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = v + shfl_xor(v, o);
  return v;
}

// Sum of squares of this thread's entries of column C (rows above `from`
// excluded), summed over the warp.
template <int C, int NPC, int R, class T>
__device__ __forceinline__ T col_norm2(const T (&a)[R][NPC], int rbase, int from) {
  if constexpr (std::is_same<T, df64>::value) {
    df64_acc acc;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const T v = (rbase + 32 * q >= from) ? a[q][C] : T(0);
      acc.add_prod(v, v);
    }
    return warp_sum(acc.value());
  } else {
    T ss = T(0);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const T v = (rbase + 32 * q >= from) ? a[q][C] : T(0);
      ss = fma(v, v, ss);
    }
    return warp_sum(ss);
  }
}

// Phase A of a column: s[c] = sum over the thread's rows of x_q a[q][c]
// (x is zero above the pivot row, so those rows add nothing).
template <int NPC, int R, class T>
__device__ __forceinline__ void column_dots(const T (&a)[R][NPC], const T* xcur, int rbase, T (&s)[NPC]) {
  if constexpr (std::is_same<T, df64>::value) {
    df64_acc acc[NPC];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const T xq = xcur[rbase + 32 * q];
#pragma unroll
      for (int c = 0; c < NPC; ++c) acc[c].add_prod(xq, a[q][c]);
    }
#pragma unroll
    for (int c = 0; c < NPC; ++c) s[c] = acc[c].value();
  } else {
#pragma unroll
    for (int c = 0; c < NPC; ++c) s[c] = T(0);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const T xq = xcur[rbase + 32 * q];
#pragma unroll
      for (int c = 0; c < NPC; ++c) s[c] = fma(xq, a[q][c], s[c]);
    }
  }
}

// The dot products of column_dots for the local columns c >= C0 only (the
// others are set to zero): the R-only form needs no Gram entries, so the
// columns at or left of the pivot (Householder vectors) are skipped.
template <int C0, int NPC, int R, class T>
__device__ __forceinline__ void column_dots_from(const T (&a)[R][NPC], const T* xcur, int rbase, T (&s)[NPC]) {
#pragma unroll
  for (int c = 0; c < NPC; ++c) s[c] = T(0);
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const T xq = xcur[rbase + 32 * q];
#pragma unroll
    for (int c = C0; c < NPC; ++c) s[c] = fma(xq, a[q][c], s[c]);
  }
}

// column_dots / column_dots_from with the thread's entries of x_j through an
// accessor xr(q) (registers or shared memory, see tile_update_la_x).
template <int NPC, int R, class T, class X>
__device__ __forceinline__ void column_dots_x(const T (&a)[R][NPC], X xr, T (&s)[NPC]) {
  if constexpr (std::is_same<T, df64>::value) {
    df64_acc acc[NPC];
#pragma unroll
    for (int q = 0; q < R; ++q)
#pragma unroll
      for (int c = 0; c < NPC; ++c) acc[c].add_prod(xr(q), a[q][c]);
#pragma unroll
    for (int c = 0; c < NPC; ++c) s[c] = acc[c].value();
  } else {
#pragma unroll
    for (int c = 0; c < NPC; ++c) s[c] = T(0);
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const T xq = xr(q);
#pragma unroll
      for (int c = 0; c < NPC; ++c) s[c] = fma(xq, a[q][c], s[c]);
    }
  }
}
template <int C0, int NPC, int R, class T, class X>
__device__ __forceinline__ void column_dots_from_x(const T (&a)[R][NPC], X xr, T (&s)[NPC]) {
#pragma unroll
  for (int c = 0; c < NPC; ++c) s[c] = T(0);
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const T xq = xr(q);
#pragma unroll
    for (int c = C0; c < NPC; ++c) s[c] = fma(xq, a[q][c], s[c]);
  }
}

// Trailing update of the thread's tile for column j, with the first trailing
// local column C0 known at compile time: a[q][c] -= d[c] x_q for c >= C0.
// The thread's rows are rbase + 32 q (q < R); the published pivot column x_j
// is zero above row j, so the update needs no row test.  The warp owning
// column j (local index C0 - 1) stores v_j = x scal below the pivot; the warp
// owning column j + 1 (local index C0) publishes it, zeroed above row j + 1,
// and its squared norm over this row group (look-ahead: the reflector of
// column j + 1 is formed from it before column j + 1's dot products).
template <int C0, int NPC, int R, class T>
__device__ __forceinline__ void tile_update(T (&a)[R][NPC], const T (&d)[NPC], const T* xcur, T* xnext, int j,
                                            int rbase, bool own_j, bool own_next, T scal, T* nnext) {
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const T xq = xcur[rbase + 32 * q];
#pragma unroll
    for (int c = C0; c < NPC; ++c) a[q][c] = fma(-d[c], xq, a[q][c]);
  }
  if constexpr (C0 >= 1) {
    if (own_j) {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int r = rbase + 32 * q;
        if (r > j) a[q][C0 - 1] = xcur[r] * scal;
      }
    }
  }
  if constexpr (C0 < NPC) {
    if (own_next) {
#pragma unroll
      for (int q = 0; q < R; ++q) xnext[rbase + 32 * q] = (rbase + 32 * q > j) ? a[q][C0] : T(0);
      const T ss = col_norm2<C0, NPC, R>(a, rbase, j + 1);
      if ((threadIdx.x & 31) == 0) *nnext = ss;
    }
  }
}

// Look-ahead form of tile_update for a tile held by one row group (every warp
// holds all rows of its columns).  The warp owning column j + 1 updates that
// column first, publishes x_{j+1} (zero above row j + 1), forms reflector
// j + 1 from its squared norm and a_{j+1,j+1} (every lane, no broadcast),
// stores the scalars in `refl_next` and arrives on the named barrier
// `bar_next`; only then does it update its other trailing columns.  The other
// warps can start column j + 1 while it finishes column j.  xr(q): this
// thread's entry of x_j in register row q (from registers where the tile
// leaves room for them, else from shared memory).
template <int C0, int NPC, int R, class T, class X>
__device__ __forceinline__ void tile_update_la_x(T (&a)[R][NPC], const T (&d)[NPC], X xr, T* xnext, int j,
                                               int rbase, bool own_j, bool own_next, T scal, T* refl_next,
                                               T* taus, int bar_next, int nthreads) {
  if constexpr (C0 < NPC) {
    if (own_next) {
#pragma unroll
      for (int q = 0; q < R; ++q) a[q][C0] = fma(-d[C0], xr(q), a[q][C0]);
#pragma unroll
      for (int q = 0; q < R; ++q) xnext[rbase + 32 * q] = (rbase + 32 * q > j) ? a[q][C0] : T(0);
      const T ss = col_norm2<C0, NPC, R>(a, rbase, j + 1);
      // a_{j+1,j+1}: register row (j + 1) / 32 < 4 of lane (j + 1) % 32
      T al = T(0);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (rbase + 32 * q == j + 1) al = a[q][C0];
      const Reflector<T> f = make_reflector(ss, shfl_from(al, (j + 1) & 31));
      if ((threadIdx.x & 31) == 0) {
        refl_next[0] = f.beta;
        refl_next[1] = f.scal;
        refl_next[2] = f.ib;
        refl_next[3] = f.tau;
        refl_next[4] = f.ident ? T(1) : T(0);
        taus[j + 1] = f.tau;
      }
      __syncwarp();
      named_bar_arrive(bar_next, nthreads);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const T xq = xr(q);
#pragma unroll
        for (int c = C0 + 1; c < NPC; ++c) a[q][c] = fma(-d[c], xq, a[q][c]);
      }
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const T xq = xr(q);
#pragma unroll
        for (int c = C0; c < NPC; ++c) a[q][c] = fma(-d[c], xq, a[q][c]);
      }
    }
  }
  if constexpr (C0 >= 1) {
    if (own_j) {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int r = rbase + 32 * q;
        if (r > j) a[q][C0 - 1] = xr(q) * scal;
      }
    }
  }
}

// Calls f(std::integral_constant<int, C>()) with C = min(c0, NPC): the first
// trailing local column of a column step, as a compile-time constant for
// the register-tile updates (c0 >= 0, warp-uniform).
template <int NPC, int C = 0, class F>
__device__ __forceinline__ void with_c0(int c0, F&& f) {
  if constexpr (C >= NPC) {
    f(std::integral_constant<int, NPC>());
  } else {
    if (c0 == C) f(std::integral_constant<int, C>());
    else with_c0<NPC, C + 1>(c0, f);
  }
}

// Y between Step 1 and Step 3 is kept in the compute format when that has the
// storage's size (double-float pairs in place of binary64): no conversion.
template <class S, class T>
using YStore = typename std::conditional<std::is_same<T, df64>::value, df64, S>::type;

// ---------------------------------------------------------------------------
// Step 1: local Householder QR of one row block per CTA.
//   A    : m x n row-major (storage S); block i = rows [i*b, min(i*b+b, m)).
//   Y    : output, same shape; may alias A (each tile is staged first).  NULL
//          = R-only mode (no Y, no T).
//   Rst  : p blocks of n x n binary64 (R_i, upper triangular, raw signs).
//   Tst  : kt slots of n x n binary64 per block (slot i*kt + t for tile t)
//          receiving tau_j on the diagonal and the Gram entries v_i^T v_j
//          above it (k_build_t then forms T), or NULL.
// A block taller than the register tile (b > B rows) is factored as a flat
// tree inside the CTA (the sequential reduction order of Sec. II-B / Alg. 2
// with one R carried along): tile 0 is the block's first B rows; tile t >= 1
// stacks the running R on the next bt rows and factors [R; A_t] =
// Q_t [R'; 0].  The rows of R below its diagonal are zero and stay exactly
// zero, so the Householder vectors of tile t are [I; V_t] and only V_t is
// stored (over A_t's rows of Y).
// LA (look-ahead form) is launched exactly when NRG == 1.
// GRAM = false (look-ahead form, binary64 / binary32 compute): the dot
// products that only give Gram entries (about a third of the column loop's
// FMAs) are skipped; R is the same bit for bit.  With Y == NULL this is the
// R-only form; with Y, the vectors and tau are written and the Gram entries
// are left to k_gram_oz (the tensor-core Gram of the Ozaki form).
// Launch: blockDim = 32*CS*NRG <= MAXT, gridDim = p, dynamic smem = LocalQrSmem.
// ---------------------------------------------------------------------------
template <class S, class T, int NPC, int R, int MAXT, bool LA, bool GRAM = true>
__global__ void __launch_bounds__(MAXT, 1) k_local_qr(const S* __restrict__ A, int64_t m, int n, int b, int bt,
                                                       int kt, int CS, int NRG, S* Y, double* __restrict__ Rst,
                                                       double* __restrict__ Tst, int32_t* status) {
  static_assert(R >= 4, "rows < 128 must lie in row group 0");
  static_assert(GRAM || (LA && !std::is_same<T, df64>::value), "the R-only form is the binary look-ahead loop");
  constexpr int QH = 4;  // register rows that can hold rows < n (n <= 128)
  extern __shared__ __align__(128) unsigned char smem[];
  const int NT = blockDim.x;
  const int NW = NT >> 5;
  const int B = 32 * NRG * R;
  const int NPAD = NPC * CS;
  const LocalQrSmem L(B, n, NW, NPAD, sizeof(S), sizeof(T));
  S* stage = reinterpret_cast<S*>(smem + L.stage);
  T* gram = reinterpret_cast<T*>(smem + L.stage);  // reused during the loop
  T* red = reinterpret_cast<T*>(smem + L.red);
  // pivot column, pivot row and the partial sums are double-buffered by the
  // parity of j: while slow warps still read step j's values, fast ones
  // publish step j+1's, so one barrier per phase suffices
  T* xbuf = reinterpret_cast<T*>(smem + L.xcol);
  T* piv = reinterpret_cast<T*>(smem + L.piv);
  T* taus = reinterpret_cast<T*>(smem + L.tau);
  T* refl = reinterpret_cast<T*>(smem + L.refl);  // beta, scal, 1/beta, tau, identity flag
  T* nrm = reinterpret_cast<T*>(smem + L.nrm);    // look-ahead squared norms, 2 x 32
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cs = warp % CS, rg = warp / CS;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * b;
  const int rows = static_cast<int>(m - row0 < b ? m - row0 : b);
  const int ntiles = rows <= B ? 1 : 1 + (rows - B + bt - 1) / bt;
  // thread rows: row group rg holds rows [32 R rg, 32 R (rg + 1)); lane l of
  // it holds rows 32 R rg + l + 32 q, so every row offset is a constant
  const int rbase = rg * 32 * R + lane;

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t parity = 0;
  int scale_exp = 0;
  T a[R][NPC];
  for (int t = 0; t < ntiles; ++t) {
    // tile t: data rows [tr0, tr0 + cnt) of the block in register rows
    // [off, off + cnt); register rows < off hold the running R
    const int tr0 = t == 0 ? 0 : B + (t - 1) * bt;
    const int cnt = t == 0 ? (rows < B ? rows : B) : (rows - tr0 < bt ? rows - tr0 : bt);
    const int off = t == 0 ? 0 : n;
    if (!cta_load_bulk(stage, A + (row0 + tr0) * n, static_cast<int64_t>(cnt) * n, bar, parity, status)) return;

    // Double-float compute: scale the data by a power of two (exact) chosen
    // from the largest binary64 exponent seen so far in the block, so that
    // entries are below 1 and products of small entries stay in binary32
    // range; when a tile raises it, the running R is rescaled (exact).  Y and
    // T are invariant under the scaling; R is unscaled on output.
    if constexpr (std::is_same<T, df64>::value) {
      int emax = 0;
      for (int idx = tid; idx < cnt * n; idx += NT) {
        const int ex = static_cast<int>(
            (static_cast<unsigned long long>(__double_as_longlong(static_cast<double>(stage[idx]))) >> 52) & 0x7ff);
        emax = ex != 0x7ff && ex > emax ? ex : emax;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
      int* wmax = reinterpret_cast<int*>(red);
      if (lane == 0) wmax[warp] = emax;
      __syncthreads();
      int bm = 0;
      for (int w = 0; w < NW; ++w) bm = max(bm, wmax[w]);
      const int se = bm > 0 ? bm - 1022 : 0;  // max |a| * 2^-se < 1
      if (t == 0) {
        scale_exp = se;
      } else if (se > scale_exp) {
#pragma unroll
        for (int q = 0; q < QH; ++q)
#pragma unroll
          for (int c = 0; c < NPC; ++c) a[q][c] = scale2(a[q][c], scale_exp - se);
        scale_exp = se;
      }
      __syncthreads();  // wmax (in the partial-sum buffer) is read by all
    }
    {
      // row pointer advanced by 32 rows per step: no per-row address registers
      // (with R x NPC addresses live the register tile would spill)
      const S* rp = stage + (rbase - off) * n + cs;
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int r = rbase + 32 * q - off;  // data row of the tile
        if (q >= QH || t == 0 || r >= 0) {
#pragma unroll
          for (int c = 0; c < NPC; ++c) {
            const int k = cs + c * CS;
            a[q][c] = (r < cnt && k < n) ? to_compute<T>(rp[c * CS], scale_exp) : T(0);
          }
        }
        rp += 32 * n;
      }
    }
    __syncthreads();  // stage is reused for the Gram matrix from here on

    // publish pivot column 0 (and its squared norm per row group) and pivot row 0
    if (cs == 0) {
#pragma unroll
      for (int q = 0; q < R; ++q) xbuf[rbase + 32 * q] = a[q][0];
      const T ss = col_norm2<0, NPC, R>(a, rbase, 0);
      if (lane == 0) nrm[rg] = ss;
      if (LA) {
        // one row group: reflector 0 is formed here (the look-ahead loop
        // below has no barrier for column 0)
        const Reflector<T> f0 = make_reflector(ss, shfl_from(a[0][0], 0));
        if (lane == 0) {
          refl[0] = f0.beta;
          refl[1] = f0.scal;
          refl[2] = f0.ib;
          refl[3] = f0.tau;
          refl[4] = f0.ident ? T(1) : T(0);
          taus[0] = f0.tau;
        }
      }
    }
    if (rg == 0 && lane == 0) {
#pragma unroll
      for (int c = 0; c < NPC; ++c) piv[cs + c * CS] = a[0][c];
    }
    __syncthreads();

    if constexpr (LA) {
      // ---- one row group: every warp holds all rows of its columns, so its
      //      dot products are complete after a warp reduction and only x_j
      //      and reflector j cross warps.  One named barrier per column
      //      (ids 1 and 2 by the parity of j): the owner of column j arrives
      //      once it has published them (during column j - 1), the other
      //      warps wait.  There is no end-of-column CTA barrier, so a warp
      //      may run one column ahead of the slowest: x_j is triple-buffered
      //      and the reflector scalars double-buffered, so nothing is
      //      overwritten before every warp has finished with it.
      int jb3 = 0;  // j mod 3
      // this warp's next own column jn = cs + c0 CS and its count c0 of own
      // columns at or left of the pivot, stepped per column (warp-uniform; no
      // division or modulo by CS in the loop)
      int jn = cs, c0 = 0;
      for (int j = 0; j < n; ++j) {
        const int jb = j & 1;
        const int jn3 = jb3 == 2 ? 0 : jb3 + 1;
        const T* xcur = xbuf + jb3 * B;   // x_j
        T* xnext = xbuf + jn3 * B;        // x_{j+1}
        const T* pcur = piv + jb * NPAD;  // row j (this warp's columns)
        T* pnext = piv + (jb ^ 1) * NPAD;
        T* rcur = red + jb * NW * 32;     // this warp's column sums
        const bool owner = (j == jn);
        if (owner) {
          ++c0;
          jn += CS;
        }
        if (j > 0 && !owner) named_bar_sync(1 + jb, NT);
        const T* rf = refl + jb * 8;
        Reflector<T> f;
        f.beta = rf[0];
        f.scal = rf[1];
        f.ib = rf[2];
        f.tau = rf[3];
        f.ident = rf[4] != T(0);

        // phase A: s = x_j^T A for this warp's columns (R-only: the columns
        //      right of the pivot only)
        // this thread's entries of x_j: read once and kept in registers for
        // the update in binary32 where the tile leaves room (R NPC values of
        // at most 400 bytes, at most 384 threads: 168 registers a thread),
        // else read from shared memory at each use (the binary64 loop is
        // bound by the binary64 unit, not by its loads)
        constexpr bool kXr = std::is_same<T, float>::value && R * NPC * sizeof(T) <= 400 && MAXT <= 384;
        T xv[kXr ? R : 1];
        if constexpr (kXr) {
#pragma unroll
          for (int q = 0; q < R; ++q) xv[q] = xcur[rbase + 32 * q];
        }
        auto xr = [&](int q) -> T {
          if constexpr (kXr) return xv[q];
          else return xcur[rbase + 32 * q];
        };
        {
          T s[NPC];
          if constexpr (GRAM) {
            column_dots_x(a, xr, s);
          } else {
            with_c0<NPC>(c0, [&](auto ic) { column_dots_from_x<decltype(ic)::value, NPC, R, T>(a, xr, s); });
          }
          TransposeReduce<NPC, 16>::run(s, lane, 0, NPC, rcur + warp * 32);
        }
        __syncwarp();

        // phase B: as in the general loop, with one row group; R's row j
        //      goes to shared memory, transposed into the Gram buffer's lower
        //      triangle (entry (c, j) = r_jc, c >= j; the Gram entries sit
        //      at (k, j), k < j), and back into the register rows < n once
        //      the tile is done: row j's registers are not read again within
        //      the tile (x is zero there for every later column)
        T dl = T(0);  // lane c's update coefficient d_c (broadcast per trailing column below)
        {
          const int mycol = cs + lane * CS;
          if (lane < NPC && mycol < n) {
            const T Sc = rcur[warp * 32 + lane];
            const T pc = pcur[mycol];
            if (mycol > j) {
              const T rl = Sc * f.ib;
              dl = (pc - rl) * f.scal;
              gram[mycol * n + j] = f.ident ? pc : rl;
            } else if (mycol == j) {
              gram[mycol * n + j] = f.beta;
            } else if (GRAM) {
              gram[mycol * n + j] = f.scal * (Sc - f.beta * pc);
            }
          }
        }

        // phase C: trailing update with the look-ahead of column j + 1 (the
        // coefficients of the trailing local columns only are broadcast)
        const bool own_next = (j + 1 < n) && (j + 1 == jn);
        T* rfn = refl + (jb ^ 1) * 8;
        const int bn = 1 + (jb ^ 1);
        with_c0<NPC>(c0, [&](auto ic) {
          constexpr int C0 = decltype(ic)::value;
          T d[NPC];
#pragma unroll
          for (int c = 0; c < NPC; ++c) d[c] = c >= C0 ? shfl_from(dl, c) : T(0);
          tile_update_la_x<C0, NPC, R, T>(a, d, xr, xnext, j, rbase, owner, own_next, f.scal, rfn, taus, bn, NT);
        });
        if (j + 1 < n) {
          // row j + 1 is register row (j + 1) / 32 (warp-uniform) of lane
          // (j + 1) % 32 (one row group: rbase = lane)
          const int qn = (j + 1) >> 5;
#pragma unroll
          for (int q = 0; q < QH; ++q)
            if (q == qn && lane == ((j + 1) & 31)) {
#pragma unroll
              for (int c = 0; c < NPC; ++c) pnext[cs + c * CS] = a[q][c];
            }
        }
        __syncwarp();
        jb3 = jn3;
      }
      __syncthreads();  // gram, R's rows and taus are read CTA-wide below
      // R's rows back into the register rows < n (their entries on and above
      // the diagonal; below it they hold Y's vectors, or the zeros of a
      // carried R)
#pragma unroll
      for (int q = 0; q < QH; ++q) {
        const int r = rbase + 32 * q;
        if (r < n) {
#pragma unroll
          for (int c = 0; c < NPC; ++c) {
            const int col = cs + c * CS;
            if (col >= r && col < n) a[q][c] = gram[col * n + r];
          }
        }
      }
    } else {
      // this warp's next own column jn and its count c0 of own columns at or
      // left of the pivot, stepped per column (as in the look-ahead loop)
      int jn = cs, c0 = 0;
      for (int j = 0; j < n; ++j) {
        const int jb = j & 1;
        const bool own_j = (j == jn);
        if (own_j) {
          ++c0;
          jn += CS;
        }
        const T* xcur = xbuf + jb * B;          // x_j (column j, current values)
        T* xnext = xbuf + (jb ^ 1) * B;         // x_{j+1}
        const T* pcur = piv + jb * NPAD;        // row j
        T* pnext = piv + (jb ^ 1) * NPAD;       // row j+1
        T* rcur = red + jb * NW * 32;           // partial sums of this step
        const T* ncur = nrm + jb * 32;          // squared norm of x_j per row group
        T* nnext = nrm + (jb ^ 1) * 32;         // ... of x_{j+1}

        // ---- the reflector of column j, from the look-ahead squared norm of x_j
        //      and alpha = a_jj: formed by the warp of row group 0 that owns
        //      column j, published before its dot products so that its scalar
        //      sequence overlaps the other warps' phase A
        Reflector<T> f;
        const bool owner = (rg == 0) && own_j;
        if (owner) {
          if (lane == 0) {
            T Sj = T(0);
            for (int g = 0; g < NRG; ++g) Sj += ncur[g];
            f = make_reflector(Sj, pcur[j]);
            refl[0] = f.beta;
            refl[1] = f.scal;
            refl[2] = f.ib;
            refl[3] = f.tau;
            refl[4] = f.ident ? T(1) : T(0);
            taus[j] = f.tau;
          }
          __syncwarp();
          if (NRG == 1) named_bar_arrive(1, NT);  // producer: the scalars are out
          f.beta = shfl_bcast(f.beta);
          f.scal = shfl_bcast(f.scal);
          f.ib = shfl_bcast(f.ib);
          f.tau = shfl_bcast(f.tau);
          f.ident = __shfl_sync(0xffffffffu, f.ident ? 1 : 0, 0) != 0;
        }

        // ---- phase A: s = x_j^T A over the thread's rows (rows < j give 0), CTA partials
        {
          T s[NPC];
          column_dots(a, xcur, rbase, s);
          TransposeReduce<NPC, 16>::run(s, lane, 0, NPC, rcur + warp * 32);
        }
        // one row group: each warp's column sums are its own (a warp sync
        // suffices) and only the reflector crosses warps; several row groups:
        // the partial sums cross warps too
        if (NRG == 1) {
          __syncwarp();
          if (!owner) named_bar_sync(1, NT);
        } else {
          __syncthreads();
        }
        if (!owner) {
          f.beta = refl[0];
          f.scal = refl[1];
          f.ib = refl[2];
          f.tau = refl[3];
          f.ident = refl[4] != T(0);
        }

        // ---- phase B: lane c < NPC sums the partials of its column c over the
        //      row groups, then forms R's r_jk = S_k / beta (r_jj = beta),
        //      d_c = (a_jk - r_jk) / (alpha - beta) and, for k < j, the Gram
        //      entry v_k^T v_j of the compact-WY T; every lane takes d and r_j
        //      by shuffle
        T d[NPC], rj[NPC];
        {
          T dl = T(0), rl = T(0);
          const int mycol = cs + lane * CS;
          if (lane < NPC && mycol < n) {
            T Sc = T(0);
            for (int g = 0; g < NRG; ++g) Sc += rcur[(g * CS + cs) * 32 + lane];
            const T pc = pcur[mycol];
            if (mycol > j) {
              rl = Sc * f.ib;
              dl = (pc - rl) * f.scal;
            } else if (mycol == j) {
              rl = f.beta;
            } else if (rg == 0) {
              gram[mycol * n + j] = f.scal * (Sc - f.beta * pc);
            }
          }
#pragma unroll
          for (int c = 0; c < NPC; ++c) {
            d[c] = shfl_from(dl, c);
            rj[c] = shfl_from(rl, c);
          }
        }

        // ---- phase C: trailing update, v_j, publish x_{j+1}; pivot row = R row j
        const bool own_next = (j + 1 < n) && (j + 1 == jn);
        with_c0<NPC>(c0, [&](auto ic) {
          tile_update<decltype(ic)::value, NPC, R>(a, d, xcur, xnext, j, rbase, own_j, own_next, f.scal, nnext + rg);
        });
        // rows j and j+1 (< n <= 128) are register rows q < 4 of row group 0:
        // the thread holding row j writes R's row j, the one holding row j+1
        // publishes it (after this step's update)
        if (!f.ident) {
#pragma unroll
          for (int q = 0; q < QH; ++q)
            if (rbase + 32 * q == j) {
#pragma unroll
              for (int c = 0; c < NPC; ++c) {
                const int col = cs + c * CS;
                if (col >= j && col < n) a[q][c] = rj[c];
              }
            }
        }
        if (j + 1 < n) {
#pragma unroll
          for (int q = 0; q < QH; ++q)
            if (rbase + 32 * q == j + 1) {
#pragma unroll
              for (int c = 0; c < NPC; ++c) pnext[cs + c * CS] = a[q][c];
            }
        }
        __syncthreads();
      }
    }

    if (Y != nullptr) {
      // ---- the Gram entries v_i^T v_j (i < j) and tau_j of the compact-WY
      //      form, binary64, into the upper triangle of the tile's T slot (the
      //      strictly lower part is never read); k_build_t turns them into T.
      //      Without the Gram dot products (GRAM = false) only tau_j is
      //      written: the Gram entries come from k_gram_oz.
      {
        double* Tout = Tst + (static_cast<int64_t>(blockIdx.x) * kt + t) * n * n;
        if constexpr (GRAM) {
          // row i by a warp, its entries kk >= i by the lanes (no division)
          for (int i = warp; i < n; i += NW)
            for (int kk = i + lane; kk < n; kk += 32)
              Tout[i * n + kk] = static_cast<double>(kk > i ? gram[i * n + kk] : taus[i]);
        } else {
          for (int i = tid; i < n; i += NT) Tout[i * n + i] = static_cast<double>(taus[i]);
        }
      }
      __syncthreads();

      // ---- the tile's rows of Y back through shared memory, bulk store
      //      (compute format for df64)
      using YS = YStore<S, T>;
      YS* ystage = reinterpret_cast<YS*>(stage);
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int r = rbase + 32 * q - off;
        if (r >= 0 && r < cnt) {
#pragma unroll
          for (int c = 0; c < NPC; ++c) {
            const int k = cs + c * CS;
            if (k < n) {
              if constexpr (std::is_same<YS, T>::value) ystage[r * n + k] = a[q][c];
              else ystage[r * n + k] = static_cast<YS>(a[q][c]);
            }
          }
        }
      }
      fence_proxy_async_smem();
      __syncthreads();
      cta_store_bulk(reinterpret_cast<YS*>(Y) + (row0 + tr0) * n, ystage, static_cast<int64_t>(cnt) * n);
    }
    if (t + 1 < ntiles) {
      // the running R for the next tile: clear what lies below its diagonal
      // (tile 0's Y_top; later tiles leave exact zeros there)
#pragma unroll
      for (int q = 0; q < QH; ++q) {
        const int r = rbase + 32 * q;
#pragma unroll
        for (int c = 0; c < NPC; ++c)
          if (r < n && cs + c * CS < r) a[q][c] = T(0);
      }
      // the stage's generic-proxy writes (Gram, Y) are ordered before the next
      // tile's bulk load, and the bulk store has read it (waited in the store)
      fence_proxy_async_smem();
      __syncthreads();
    }
  }  // tiles

  // ---- R_i (raw signs) for rows < n
#pragma unroll
  for (int q = 0; q < QH; ++q) {
    const int r = rbase + 32 * q;
    if (r < n) {
#pragma unroll
      for (int c = 0; c < NPC; ++c) {
        const int k = cs + c * CS;
        if (k < n)
          Rst[static_cast<int64_t>(blockIdx.x) * n * n + r * n + k] =
              (k >= r && r < rows) ? (scale_exp ? ldexp(static_cast<double>(a[q][c]), scale_exp)
                                                 : static_cast<double>(a[q][c]))
                                   : 0.0;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Step 3: Q_i = Q1_i C_i with C_i = Q2_i (n x n binary64), one CTA per row
// block.  A block of one tile gives Q_i = [C; 0] - Y_i W, W = T (Y_top^T C).
// A block factored as a flat tree of tiles (k_local_qr) is taken tile by
// tile, last to first, with X = C: tile t >= 1 has Householder vectors
// [I; V_t], so W_t = T_t X, its rows of Q are -V_t W_t and tile t-1 gets
// X - W_t; tile 0 is the one-tile case with C = X.
//   Yg  : m x n (storage S), as written by k_local_qr.
//   Tg  : kt slots of n x n binary64 per block (T of each tile, upper part).
//   Cg  : cblocks blocks of n x n binary64 (cblocks == 1: one C for all).
//   Qg  : output m x n (storage S); may alias Yg.
// The n x n operands stream through the stage in row chunks; each thread
// keeps its (at most kMaxE) entries of an n x NPAD product in registers.
// skew != 0: lane l takes the columns kk of its staged rows in the order
// l mod n, l mod n + 1, ... (cyclic), so that the lanes' reads of one step
// spread over the banks (the sum is the same up to rounding order).
// ---------------------------------------------------------------------------
// entries of an n x NPAD product per thread: n NPAD / (32 CS NRG) = NPC n / (32 NRG)
template <int NPC>
constexpr int max_entries() { return (NPC * 100 + 31) / 32; }  // n <= 100

template <class S, class T, int NPC, int R, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_form_q(const S* Yg, int64_t m, int n, int b, int bt, int kt, int srows,
                                                     int CS, int NRG, int skew, const double* __restrict__ Tg,
                                                     const double* __restrict__ Cg, int64_t cblocks, S* Qg,
                                                     int32_t* status) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int NT = blockDim.x;
  const int NPAD = NPC * CS;
  const int B = 32 * NRG * R;
  const FormQSmem L(srows, n, NPAD, sizeof(S), sizeof(T));
  S* stage = reinterpret_cast<S*>(smem + L.stage);
  T* Xm = reinterpret_cast<T*>(smem + L.xm);
  T* Wm = reinterpret_cast<T*>(smem + L.wm);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cs = warp % CS, rg = warp / CS;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * b;
  const int rows = static_cast<int>(m - row0 < b ? m - row0 : b);
  const int ntiles = rows <= B ? 1 : 1 + (rows - B + bt - 1) / bt;
  const int rbase = rg * 32 * R + lane;  // thread rows rbase + 32 q, as in k_local_qr
  const int ntop = rows < n ? rows : n;
  const int NE = n * NPAD;
  using YS = YStore<S, T>;
  const YS* Yb = reinterpret_cast<const YS*>(Yg) + row0 * n;
  YS* ystage = reinterpret_cast<YS*>(stage);
  T* tm = reinterpret_cast<T*>(stage);
  // rows of an n-column matrix of 8-byte values that the stage holds
  const int crow = static_cast<int>(static_cast<size_t>(srows) * sizeof(S) / 8);

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  const int64_t cb = cblocks == 1 ? 0 : static_cast<int64_t>(blockIdx.x);
  const double* Cb = Cg + cb * n * n;
  for (int idx = tid; idx < NE; idx += NT) {  // X = C
    const int kk = idx / NPAD, c = idx % NPAD;
    Xm[idx] = c < n ? to_compute<T>(Cb[kk * n + c], 0) : T(0);
  }
  __syncthreads();

  uint32_t parity = 0;
  for (int t = ntiles - 1; t >= 0; --t) {
    const int tr0 = t == 0 ? 0 : B + (t - 1) * bt;  // first row of the tile's data in the block
    const int cnt = t == 0 ? (rows < B ? rows : B) : (rows - tr0 < bt ? rows - tr0 : bt);
    const double* Tb = Tg + (static_cast<int64_t>(blockIdx.x) * kt + t) * n * n;
    constexpr int kMaxE = max_entries<NPC>();
    T w[kMaxE];
    const T* src = Xm;
    if (t == 0) {
      // Z = Y_top^T X (Y_top unit lower triangular), Y_top streamed by rows;
      // read before any row of the block is overwritten
#pragma unroll
      for (int e = 0; e < kMaxE; ++e) {
        const int idx = tid + e * NT, kk = idx / NPAD, c = idx % NPAD;
        w[e] = (idx < NE && c < n && kk < ntop) ? Xm[idx] : T(0);
      }
      for (int r0 = 0; r0 < ntop; r0 += crow) {
        const int r1 = ntop < r0 + crow ? ntop : r0 + crow;
        for (int idx = tid; idx < (r1 - r0) * n; idx += NT) ystage[idx] = Yb[static_cast<int64_t>(r0) * n + idx];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < kMaxE; ++e) {
          const int idx = tid + e * NT, kk = idx / NPAD, c = idx % NPAD;
          if (idx < NE && c < n)
            for (int r = (r0 > kk + 1 ? r0 : kk + 1); r < r1; ++r)
              w[e] = fma(static_cast<T>(ystage[(r - r0) * n + kk]), Xm[r * NPAD + c], w[e]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int e = 0; e < kMaxE; ++e)
        if (tid + e * NT < NE) Wm[tid + e * NT] = w[e];
      __syncthreads();
      src = Wm;
    }
    // W = T src (T upper triangular), T streamed by rows: row kk of W is
    // complete in the chunk that holds row kk of T
#pragma unroll
    for (int e = 0; e < kMaxE; ++e) w[e] = T(0);
    for (int k0 = 0; k0 < n; k0 += crow) {
      const int k1 = n < k0 + crow ? n : k0 + crow;
      for (int idx = tid; idx < (k1 - k0) * n; idx += NT) {
        const int i = idx / n, col = idx % n;
        tm[idx] = col >= k0 + i ? to_compute<T>(Tb[static_cast<int64_t>(k0) * n + idx], 0) : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int e = 0; e < kMaxE; ++e) {
        const int idx = tid + e * NT, kk = idx / NPAD, c = idx % NPAD;
        if (idx < NE && c < n && kk >= k0 && kk < k1)
          for (int i = kk; i < n; ++i) w[e] = fma(tm[(kk - k0) * n + i], src[i * NPAD + c], w[e]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int e = 0; e < kMaxE; ++e) {
      const int idx = tid + e * NT;
      if (idx < NE) {
        Wm[idx] = w[e];
        if (t > 0) Xm[idx] = Xm[idx] - w[e];  // coefficient of tile t-1
      }
    }
    __syncthreads();

    // the tile's rows of Q, chunk by chunk of `srows` staged rows:
    // tile 0: [X; 0] - Y W (unit lower Y_top); tile t >= 1: -V_t W
    const bool top = (t == 0);
    for (int c0 = 0; c0 < cnt; c0 += srows) {
      const int crows = cnt - c0 < srows ? cnt - c0 : srows;
      const int64_t g0 = row0 + tr0 + c0;  // first matrix row of the chunk
      if (!cta_load_bulk(ystage, reinterpret_cast<const YS*>(Yg) + g0 * n, static_cast<int64_t>(crows) * n, bar,
                         parity, status))
        return;
      T acc[R][NPC];
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int r = c0 + rbase + 32 * q;  // row within the tile
#pragma unroll
        for (int c = 0; c < NPC; ++c) {
          const int kc = cs + c * CS;
          acc[q][c] = (top && r < ntop && kc < n) ? Xm[r * NPAD + kc] : T(0);
        }
      }
      int kk = skew ? lane % n : 0;
      for (int step = 0; step < n; ++step, kk = (kk + 1 == n) ? 0 : kk + 1) {
        T wk[NPC];
#pragma unroll
        for (int c = 0; c < NPC; ++c) wk[c] = Wm[kk * NPAD + cs + c * CS];
        const YS* yp = ystage + rbase * n + kk;  // advanced by 32 rows per step
#pragma unroll
        for (int q = 0; q < R; ++q) {
          const int rl = rbase + 32 * q;  // row within the chunk
          const int r = c0 + rl;
          T y = T(0);
          if (rl < crows) y = static_cast<T>(*yp);
          if (top && kk >= r) y = (kk == r) ? T(1) : T(0);
          yp += 32 * n;
#pragma unroll
          for (int c = 0; c < NPC; ++c) acc[q][c] = fma(-y, wk[c], acc[q][c]);
        }
      }
      __syncthreads();  // every read of this chunk in shared memory is done
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int rl = rbase + 32 * q;
        if (rl < crows) {
#pragma unroll
          for (int c = 0; c < NPC; ++c) {
            const int kc = cs + c * CS;
            if (kc < n) stage[rl * n + kc] = to_storage<S>(acc[q][c]);
          }
        }
      }
      fence_proxy_async_smem();
      __syncthreads();
      cta_store_bulk(Qg + g0 * n, stage, static_cast<int64_t>(crows) * n);
      __syncthreads();  // the stage is free again (bulk store read it, tail stores done)
    }
  }
}

}  // namespace tsqr
