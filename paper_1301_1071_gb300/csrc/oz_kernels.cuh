// oz_kernels.cuh -- Step 3 (Sec. III-B: Q_i = Q1_i Q2_i) for binary64 data
// with the product Y_i W_i on the 5th-generation tensor cores, by the
// error-free splitting of Ozaki, Ogita, Oishi and Rump ("Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012), with
// binary16 tensor-core products accumulated in binary32 (the adaptation of
// Mukunoki, Ozaki, Ogita and Imamura, "DGEMM using tensor cores, and its
// accurate and reproducible versions", ISC 2020).
//
// Splitting.  Row r of a chunk of Y (K = n columns) is written relative to
// its largest binary exponent E_r as a 56-bit fixed-point integer per entry,
// |y_rk| ~ F_rk 2^(E_r - 1078) (truncated; the error is below 2^-55 of the
// row's largest entry), and F_rk is cut into S = 7 digits of B = 8 bits:
// y_rk ~ sum_s sign(y_rk) f_rks 2^(8 (S-1-s)) 2^(E_r - 1078), 0 <= f < 256.
// Column c of W is split the same way with its own exponent G_c.  Every
// digit is an integer of at most 8 bits, exact in binary16.
//
// Exact products.  For each diagonal d = s + t <= S - 1 the tensor cores form
// D_d = sum_{s+t=d} Ydigits_s Wdigits_t: at most (d+1) n terms of magnitude
// < 2^16 per entry, all integers, so for n <= 32 every partial sum is an
// integer below 7 * 32 * 2^16 < 2^24 and the binary32 accumulation is exact
// (whatever its order).  The dropped diagonals d >= S weigh below 2^-56 of the
// row-by-column scale.
//
// Recombination.  P = sum_d D_d 2^(8 (S-1-d) - 10) in a 64-bit integer (the
// lowest two diagonals shifted right, an error below 2^-60 of P's range),
// then one rounding to binary64 and an exact scaling by a power of two:
// (Y W)_rc ~ P 2^(E_r + G_c - 2098).  Apart from W's formation, no binary64
// arithmetic is spent on the product.
//
// Structure (as k_form_q): one CTA per row block; tiles last to first with
// X = C: tile t >= 1 has W_t = T_t X, its rows of Q are -V_t W_t, and X <- X -
// W_t; tile 0 has W = T (Y_top^T X) and rows [X; 0] - Y W.  W is formed in
// binary64 on the CUDA cores with the operation order of k_form_q.  The tile's
// rows go in chunks of 128 (one tensor-memory lane per row): each chunk
// arrives by bulk copy, is split into the A digits, the next chunk's copy is
// started, the 28 digit products are issued by one thread and complete on an
// mbarrier, and the epilogue reads the 7 accumulators (tcgen05.ld), recombines
// and writes the chunk's rows of Q over Y.
//
// Operand layout: binary16, K-major, no swizzle: core matrices of 8 rows x
// 16 bytes (8 values); element (r, k) at ((r/8) K/8 + k/8) 128 + (r%8) 16 +
// (k%8) 2 bytes; leading offset (next core along K) 128 bytes, stride offset
// (next 8-row group) K/8 x 128 bytes.
#pragma once

#include <cstdint>

#include "device.cuh"
#include "layout.cuh"
#include "tcgen05.cuh"

namespace tsqr {

constexpr int kOzThreads = 256;  // 8 warps
constexpr int kOzM = 128;        // rows per chunk (tensor-memory lanes)
constexpr int kOzDigits = 7;     // S
constexpr int kOzBits = 8;       // bits per digit
constexpr int kOzMaxN = 32;      // exact binary32 accumulation: 7 n 2^16 < 2^24
constexpr int kOzShift = 10;     // P = sum_d D_d 2^(8 (S-1-d) - kOzShift) fits 63 bits
constexpr int kOzMaxE = (kOzMaxN * kOzMaxN + kOzThreads - 1) / kOzThreads;  // W entries per thread

TSQR_HD constexpr int oz_k(int n) { return n <= 16 ? 16 : 32; }  // K = N, a multiple of 16
TSQR_HD constexpr int oz_tmem_cols(int K) { return kOzDigits * K <= 128 ? 128 : 256; }

// Shared-memory layout of k_form_q_oz (identical on host and device).
struct FormQOzSmem {
  size_t a, b, ys, xm, wm, rexp, cexp, bar, lbar, tslot, total;
  TSQR_HD FormQOzSmem(int n) {
    const size_t K = oz_k(n);
    size_t o = 0;
    a = o; o = align_up(o + kOzDigits * kOzM * K * 2, 128);   // A digits, 7 x 128 x K binary16
    b = o; o = align_up(o + kOzDigits * K * K * 2, 128);      // B digits, 7 x N x K binary16
    ys = o; o = align_up(o + (size_t)kOzM * n * 8, 128);      // the chunk's rows of Y (binary64)
    xm = o; o = align_up(o + (size_t)n * n * 8, 16);          // X (binary64, n x n)
    wm = o; o = align_up(o + (size_t)n * n * 8, 16);          // W (binary64, n x n)
    rexp = o; o = align_up(o + kOzM * 4, 16);                 // row exponents of the chunk
    cexp = o; o = align_up(o + K * 4, 16);                    // column exponents of W
    bar = o; o = align_up(o + 8, 8);                          // MMA completion
    lbar = o; o = align_up(o + 8, 8);                         // chunk arrival
    tslot = o; o = align_up(o + 8, 16);                       // tensor-memory address
    total = o;
  }
};

#if defined(__CUDACC__) && defined(TSQR_OZ_KERNELS)

// binary64 -> (biased exponent, 53-bit significand, sign); zero and
// subnormals take the exponent 1 (their significand has no hidden bit).
__device__ __forceinline__ void oz_unpack(double y, int& e, uint64_t& mant, uint32_t& neg) {
  const uint64_t bits = static_cast<uint64_t>(__double_as_longlong(y));
  e = static_cast<int>((bits >> 52) & 0x7FF);
  mant = bits & 0xFFFFFFFFFFFFFull;
  if (e) mant |= 1ull << 52;
  else e = 1;
  neg = static_cast<uint32_t>(bits >> 63);
}

// Two digits (0 <= f < 256) with their signs as a binary16 pair: 1024 + f has
// the bit pattern 0x6400 | f, and 1024 is subtracted exactly.
__device__ __forceinline__ uint32_t oz_half2(uint32_t f0, uint32_t f1, uint32_t n0, uint32_t n1) {
  const uint32_t biased = (0x6400u | f0) | ((0x6400u | f1) << 16);
  uint32_t h;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(h) : "r"(biased), "r"(0x64006400u));
  return h ^ ((n0 << 15) | (n1 << 31));
}

// Stores the S digits of 8 fixed-point values (one 8-wide group along K of
// one operand row): digit s of the group, as 8 binary16 values, goes to
// dst + s * slice_bytes (16 bytes).
__device__ __forceinline__ void oz_store_digits(const uint64_t (&F)[8], const uint32_t (&neg)[8], char* dst,
                                                uint32_t slice_bytes) {
#pragma unroll
  for (int s = 0; s < kOzDigits; ++s) {
    const int sh = kOzBits * (kOzDigits - 1 - s);
    uint32_t f[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) f[i] = static_cast<uint32_t>(F[i] >> sh) & 0xFFu;
    uint4 v;
    v.x = oz_half2(f[0], f[1], neg[0], neg[1]);
    v.y = oz_half2(f[2], f[3], neg[2], neg[3]);
    v.z = oz_half2(f[4], f[5], neg[4], neg[5]);
    v.w = oz_half2(f[6], f[7], neg[6], neg[7]);
    *reinterpret_cast<uint4*>(dst + s * slice_bytes) = v;
  }
}

// The 56-bit fixed-point integers of 8 values against the exponent emax.
__device__ __forceinline__ void oz_fixed(const int (&e)[8], const uint64_t (&mant)[8], int emax, uint64_t (&F)[8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int sh = emax - e[i];
    F[i] = sh >= 56 ? 0ull : ((mant[i] << 3) >> sh);
  }
}

// x 2^s, exact: an exponent-field add while the result stays normal, else
// the library's ldexp (subnormal or overflowing results).
__device__ __forceinline__ double oz_scale(double v, int s) {
  const long long bits = __double_as_longlong(v);
  const int e = static_cast<int>((bits >> 52) & 0x7FF);
  const int ne = e + s;
  if (e != 0 && ne > 0 && ne < 0x7FF) return __longlong_as_double(bits + (static_cast<long long>(s) << 52));
  return ldexp(v, s);
}

// Step 3, binary64 data, Ozaki-split tensor-core product.
//   Yg : m x n (binary64), Y as written by k_local_qr; Q is written over it.
//   Tg : kt slots of n x n binary64 per block (upper triangle).
//   Cg : cblocks blocks of n x n binary64 (cblocks == 1: one C for all).
// Launch: gridDim = p, blockDim = kOzThreads, dynamic smem = FormQOzSmem(n).
template <int K>
__global__ void __launch_bounds__(kOzThreads, 2)
    k_form_q_oz(double* Yg, int64_t m, int n, int b, int B, int bt, int kt, const double* __restrict__ Tg,
                const double* __restrict__ Cg, int64_t cblocks, int32_t* status) {
  constexpr int N = K;             // accumulator columns per diagonal
  constexpr int GPR = K / 8;       // 8-wide groups along K: threads per operand row in the split
  constexpr int NC = oz_tmem_cols(K);
  constexpr uint32_t kSliceA = kOzM * K * 2, kSliceB = N * K * 2;
  constexpr uint32_t kLbo = 128, kSbo = (K / 8) * 128;
  extern __shared__ __align__(1024) unsigned char smem[];
  const FormQOzSmem L(n);
  char* a_dig = reinterpret_cast<char*>(smem + L.a);
  char* b_dig = reinterpret_cast<char*>(smem + L.b);
  double* ys = reinterpret_cast<double*>(smem + L.ys);
  double* xm = reinterpret_cast<double*>(smem + L.xm);
  double* wm = reinterpret_cast<double*>(smem + L.wm);
  int* rexp = reinterpret_cast<int*>(smem + L.rexp);
  int* cexp = reinterpret_cast<int*>(smem + L.cexp);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
  uint64_t* lbar = reinterpret_cast<uint64_t*>(smem + L.lbar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.tslot);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nn = n * n;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * b;
  const int rows = static_cast<int>(m - row0 < b ? m - row0 : b);
  const int ntiles = rows <= B ? 1 : 1 + (rows - B + bt - 1) / bt;
  const int ntop = rows < n ? rows : n;
  const uint32_t idesc = tc_idesc_f16(kOzM, N);

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(lbar, 1);
    fence_mbar_init();
  }
  if (warp == 0) tc_alloc(tslot, NC);
  const int64_t cb = cblocks == 1 ? 0 : static_cast<int64_t>(blockIdx.x);
  for (int idx = tid; idx < nn; idx += kOzThreads) xm[idx] = Cg[cb * nn + idx];  // X = C
  // this thread's entries of an n x n product: idx = tid + e kOzThreads = kk n + c
  int ekk[kOzMaxE], ec[kOzMaxE];
#pragma unroll
  for (int e = 0; e < kOzMaxE; ++e) {
    const int idx = tid + e * kOzThreads;
    ekk[e] = idx < nn ? idx / n : n;
    ec[e] = idx < nn ? idx % n : 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  auto tile_rows = [&](int t, int& tr0, int& cnt) {
    tr0 = t == 0 ? 0 : B + (t - 1) * bt;
    cnt = t == 0 ? (rows < B ? rows : B) : (rows - tr0 < bt ? rows - tr0 : bt);
  };
  // Issue (thread 0) the bulk copy of the 16-byte-aligned body of chunk
  // (t, c0) into ys; the rest is read with plain loads on arrival.
  auto issue = [&](int t, int c0) {
    int tr0, cnt;
    tile_rows(t, tr0, cnt);
    const int crows = cnt - c0 < kOzM ? cnt - c0 : kOzM;
    const double* src = Yg + (row0 + tr0 + c0) * n;
    const uint32_t bytes = static_cast<uint32_t>(crows) * n * 8;
    const uint32_t body = (reinterpret_cast<uintptr_t>(src) & 15) == 0 ? (bytes & ~15u) : 0u;
    if (tid == 0 && body > 0) {
      mbar_arrive_expect_tx(lbar, body);
      for (uint32_t off = 0; off < body; off += kBulkChunk) {
        const uint32_t len = body - off < kBulkChunk ? body - off : kBulkChunk;
        bulk_g2s(reinterpret_cast<char*>(ys) + off, reinterpret_cast<const char*>(src) + off, len, lbar);
      }
    }
    return body;
  };

  uint32_t parity = 0, lph = 0;
  bool pend = false;  // a bulk copy into ys has not been waited for
  bool ok = true;
  int t = ntiles - 1, c0 = 0, cur_tile = -1;
  uint32_t body = issue(t, c0);
  pend = body > 0;
  for (;;) {
    int tr0, cnt;
    tile_rows(t, tr0, cnt);
    const int crows = cnt - c0 < kOzM ? cnt - c0 : kOzM;
    double* yq = Yg + (row0 + tr0 + c0) * n;  // first row of the chunk (Y in, Q out)
    const bool top = (t == 0);
    // ---- this chunk's Y: bulk body, then the plain-load remainder
    if (body > 0) {
      ok = mbar_wait_bounded(lbar, lph);
      if (ok) {
        lph ^= 1u;
        pend = false;
      }
    }
    for (int e = static_cast<int>(body / 8) + tid; e < crows * n; e += kOzThreads) ys[e] = yq[e];
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok) {
      if (tid == 0) set_status(status, TSQR_ERR_TIMEOUT);
      break;
    }
    if (t != cur_tile) {
      // ---- prologue of tile t: W (binary64, k_form_q's operation order) and
      //      its column digits
      cur_tile = t;
      const double* Tb = Tg + (static_cast<int64_t>(blockIdx.x) * kt + t) * nn;
      const double* src = xm;
      double w[kOzMaxE];
      if (t == 0) {
        // Z = Y_top^T X with Y_top unit lower triangular: rows < ntop of the
        // block, which are rows < ntop of this chunk (c0 == 0)
#pragma unroll
        for (int e = 0; e < kOzMaxE; ++e) {
          const int kk = ekk[e], c = ec[e];
          double acc = 0.0;
          if (kk < ntop) {
            acc = xm[kk * n + c];
            for (int r = kk + 1; r < ntop; ++r) acc = fma(ys[r * n + kk], xm[r * n + c], acc);
          }
          w[e] = acc;
        }
#pragma unroll
        for (int e = 0; e < kOzMaxE; ++e)
          if (ekk[e] < n) wm[ekk[e] * n + ec[e]] = w[e];
        __syncthreads();
        src = wm;
      }
      // W = T src (T upper triangular)
#pragma unroll
      for (int e = 0; e < kOzMaxE; ++e) {
        const int kk = ekk[e], c = ec[e];
        double acc = 0.0;
        if (kk < n)
          for (int i = kk; i < n; ++i) acc = fma(__ldg(Tb + kk * n + i), src[i * n + c], acc);
        w[e] = acc;
      }
      __syncthreads();
#pragma unroll
      for (int e = 0; e < kOzMaxE; ++e) {
        if (ekk[e] < n) {
          const int idx = ekk[e] * n + ec[e];
          wm[idx] = w[e];
          if (t > 0) xm[idx] -= w[e];  // coefficient of tile t-1
        }
      }
      __syncthreads();
      // B digits: operand row c (= column c of W), 8-wide group g along K
      if (tid < N * GPR) {
        const int c = tid / GPR, g = tid % GPR;
        int e[8];
        uint64_t mant[8];
        uint32_t neg[8];
        int emax = 1;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = 8 * g + i;
          const double v = (c < n && k < n) ? wm[k * n + c] : 0.0;
          oz_unpack(v, e[i], mant[i], neg[i]);
          if (mant[i] != 0 && e[i] > emax) emax = e[i];
        }
#pragma unroll
        for (int o = 1; o < GPR; o <<= 1) {
          const int other = __shfl_xor_sync(0xffffffffu, emax, o);
          emax = other > emax ? other : emax;
        }
        if (g == 0) cexp[c] = emax;
        uint64_t F[8];
        oz_fixed(e, mant, emax, F);
        oz_store_digits(F, neg, b_dig + ((c / 8) * (K / 8) + g) * 128 + (c % 8) * 16, kSliceB);
      }
    }
    // ---- A digits of the chunk's rows (tile 0: the unit lower Y_top)
#pragma unroll
    for (int pass = 0; pass < kOzM * GPR / kOzThreads; ++pass) {
      const int r = pass * (kOzThreads / GPR) + tid / GPR, g = tid % GPR;
      int e[8];
      uint64_t mant[8];
      uint32_t neg[8];
      int emax = 1;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = 8 * g + i;
        double y = 0.0;
        if (r < crows && k < n) {
          y = ys[r * n + k];
          if (top && c0 + r < ntop && k >= c0 + r) y = (k == c0 + r) ? 1.0 : 0.0;
        }
        oz_unpack(y, e[i], mant[i], neg[i]);
        if (mant[i] != 0 && e[i] > emax) emax = e[i];
      }
#pragma unroll
      for (int o = 1; o < GPR; o <<= 1) {
        const int other = __shfl_xor_sync(0xffffffffu, emax, o);
        emax = other > emax ? other : emax;
      }
      if (g == 0) rexp[r] = emax;
      uint64_t F[8];
      oz_fixed(e, mant, emax, F);
      oz_store_digits(F, neg, a_dig + ((r / 8) * (K / 8) + g) * 128 + (r % 8) * 16, kSliceA);
    }
    fence_proxy_async_smem();  // digit writes -> tensor-core reads; ys reads -> next bulk copy
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // ---- prefetch the next chunk into ys (every read of ys is done)
    int nt = t, nc0 = c0 + kOzM;
    if (nc0 >= cnt) {
      nt = t - 1;
      nc0 = 0;
    }
    const uint32_t body_next = nt >= 0 ? issue(nt, nc0) : 0u;
    pend = body_next > 0;
    // ---- the digit products: diagonal d accumulates s + t = d
    if (tid == 0) {
      const uint32_t a0 = smem_u32(a_dig), b0 = smem_u32(b_dig);
#pragma unroll 1
      for (int d = 0; d < kOzDigits; ++d)
#pragma unroll 1
        for (int s = 0; s <= d; ++s)
#pragma unroll
          for (int kb = 0; kb < K / 16; ++kb) {
            const uint64_t da = tc_smem_desc(a0 + s * kSliceA + kb * 256, kLbo, kSbo);
            const uint64_t db = tc_smem_desc(b0 + (d - s) * kSliceB + kb * 256, kLbo, kSbo);
            tc_mma_f16(tmem + static_cast<uint32_t>(d * N), da, db, idesc, (s > 0 || kb > 0) ? 1 : 0);
          }
      tc_commit(bar);
    }
    ok = __syncthreads_and(mbar_wait_bounded(bar, parity) ? 1 : 0) != 0;  // uniform over the CTA
    parity ^= 1u;
    tc_fence_after();
    if (!ok) {
      if (tid == 0) set_status(status, TSQR_ERR_TIMEOUT);
      break;
    }
    // ---- epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. (the
    //      chunk's rows) and the 8-column groups w / 4, w / 4 + 2, ...
    {
      const int q = warp & 3;
      const int r = 32 * q + lane;
      const int rt = c0 + r;
      const int emax = rexp[r];
      for (int g = warp >> 2; g < N / 8; g += kOzThreads / 128) {
        uint32_t v[kOzDigits][8];
#pragma unroll
        for (int d = 0; d < kOzDigits; ++d)
          tc_ld_x8(tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(d * N + 8 * g), v[d]);
        tc_wait_ld();
        if (r < crows) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int col = 8 * g + i;
            if (col < n) {
              long long P = 0;
#pragma unroll
              for (int d = 0; d < kOzDigits; ++d) {
                const long long D = static_cast<long long>(__float2int_rz(__uint_as_float(v[d][i])));
                const int sh = kOzBits * (kOzDigits - 1 - d) - kOzShift;
                P += sh >= 0 ? (D << sh) : (D >> -sh);
              }
              const double yw = P == 0 ? 0.0 : oz_scale(__ll2double_rn(P), emax + cexp[col] - 2098);
              yq[r * n + col] = (top && rt < ntop) ? xm[rt * n + col] - yw : -yw;
            }
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();  // tensor memory read before the next chunk's products
    tc_fence_after();
    if (nt < 0) break;
    t = nt;
    c0 = nc0;
    body = body_next;
  }
  // a copy still in flight after an error: wait for it (bounded) before the
  // shared memory is released
  if (!ok && pend) mbar_wait_bounded(lbar, lph);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, NC);
}

#endif  // __CUDACC__ && TSQR_OZ_KERNELS

}  // namespace tsqr
