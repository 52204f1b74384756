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
// then one rounding to binary64 with the exact power-of-two scale folded into
// the exponent: (Y W)_rc ~ P 2^(E_r + G_c - 2098), formed with integer
// operations.  Apart from W's formation, no binary64 arithmetic is spent on
// the product.
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

// Stores the S digits of 8 fixed-point values F (one 8-wide group along K of
// one operand row): digit s of the group, as 8 binary16 values, goes to
// dst + s * slice_bytes (16 bytes).  The digits are the bytes 6 - s of F, so
// a pair of values takes one byte permute (the two bytes into the low bytes
// of the two halves), one logic op (the binary16 pattern 0x6400 | f of
// 1024 + f), one exact half2 subtraction of 1024 and the sign bits.
__device__ __forceinline__ void oz_store_digits(const uint64_t (&F)[8], const uint32_t (&neg)[8], char* dst,
                                                uint32_t slice_bytes) {
  uint32_t lo[8], hi[8], sg[4];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    lo[i] = static_cast<uint32_t>(F[i]);
    hi[i] = static_cast<uint32_t>(F[i] >> 32);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) sg[j] = (neg[2 * j] << 15) | (neg[2 * j + 1] << 31);
#pragma unroll
  for (int s = 0; s < kOzDigits; ++s) {
    const int byte = kOzDigits - 1 - s;          // byte of F holding digit s
    const int jb = byte & 3;                      // ... within its 32-bit word
    const uint32_t sel = static_cast<uint32_t>(jb | ((4 + jb) << 8));
    uint32_t h[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t wa = byte >= 4 ? hi[2 * j] : lo[2 * j];
      const uint32_t wb = byte >= 4 ? hi[2 * j + 1] : lo[2 * j + 1];
      const uint32_t biased = (__byte_perm(wa, wb, sel) & 0x00FF00FFu) | 0x64006400u;
      uint32_t d;
      asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(biased), "r"(0x64006400u));
      h[j] = d ^ sg[j];
    }
    *reinterpret_cast<uint4*>(dst + s * slice_bytes) = make_uint4(h[0], h[1], h[2], h[3]);
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

// -P 2^s as binary64 for a nonzero 64-bit integer P, rounded to nearest
// (ties to even) with integer operations only: the leading bit fixes the
// exponent, a P of at most 53 significant bits is exact, a longer one is
// rounded on its dropped bits.  A result outside the normal range goes
// through the library's ldexp.
__device__ __forceinline__ double oz_neg_scaled(long long P, int s) {
  const uint64_t neg = P < 0 ? 0ull : 1ull;  // sign of -P
  uint64_t a = P < 0 ? static_cast<uint64_t>(-P) : static_cast<uint64_t>(P);
  int msb = 63 - __clzll(static_cast<long long>(a));
  uint64_t mant;
  if (msb <= 52) {
    mant = a << (52 - msb);
  } else {
    const int sh = msb - 52;
    uint64_t q = a >> sh;
    const uint64_t rem = a & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    q += (rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull;
    if (q >> 53) {
      q >>= 1;
      ++msb;
    }
    mant = q;
  }
  const int e = msb + s + 1023;
  if (e <= 0 || e >= 0x7FF) return -ldexp(static_cast<double>(P), s);
  return __longlong_as_double(static_cast<long long>((neg << 63) | (static_cast<uint64_t>(e) << 52) |
                                                     (mant & 0xFFFFFFFFFFFFFull)));
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
    // ---- the previous chunk's Q rows have left the A-digit region (thread 0's
    //      bulk store; ordered before the region's reuse by the barrier below)
    if (tid == 0) bulk_wait_read();
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
      // T of the tile into the A-digit region (idle until this chunk's split)
      double* ts = reinterpret_cast<double*>(a_dig);
      {
        const double* Tb = Tg + (static_cast<int64_t>(blockIdx.x) * kt + t) * nn;
        for (int idx = tid; idx < nn; idx += kOzThreads) ts[idx] = Tb[idx];
      }
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
        src = wm;
      }
      __syncthreads();  // T staged (and Z written)
      // W = T src (T upper triangular)
#pragma unroll
      for (int e = 0; e < kOzMaxE; ++e) {
        const int kk = ekk[e], c = ec[e];
        double acc = 0.0;
        if (kk < n)
          for (int i = kk; i < n; ++i) acc = fma(ts[kk * n + i], src[i * n + c], acc);
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
        const int c = (tid / (8 * GPR)) * 8 + (tid & 7), g = (tid >> 3) % GPR;
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
        for (int o = 8; o < 8 * GPR; o <<= 1) {
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
      const int r = pass * (kOzThreads / GPR) + (tid / (8 * GPR)) * 8 + (tid & 7), g = (tid >> 3) % GPR;
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
      for (int o = 8; o < 8 * GPR; o <<= 1) {
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
      // straight-line issue: each descriptor is the base descriptor plus the
      // operand's byte offset >> 4 in its (14-bit) address field
      const uint64_t da0 = tc_smem_desc(smem_u32(a_dig), kLbo, kSbo);
      const uint64_t db0 = tc_smem_desc(smem_u32(b_dig), kLbo, kSbo);
#pragma unroll
      for (int d = 0; d < kOzDigits; ++d)
#pragma unroll
        for (int s = 0; s <= d; ++s)
#pragma unroll
          for (int kb = 0; kb < K / 16; ++kb)
            tc_mma_f16(tmem + static_cast<uint32_t>(d * N), da0 + ((s * kSliceA + kb * 256) >> 4),
                       db0 + (((d - s) * kSliceB + kb * 256) >> 4), idesc, (s > 0 || kb > 0) ? 1 : 0);
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
    //      chunk's rows) and the 8-column groups w / 4, w / 4 + 2, ...; the
    //      chunk's rows of Q are staged in the A-digit region (free once the
    //      products completed) and leave by one bulk store
    double* qs = reinterpret_cast<double*>(a_dig);
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
              // -(Y W)_rc = -P 2^(E_r + G_c - 2098)
              const double myw = P == 0 ? 0.0 : oz_neg_scaled(P, emax + cexp[col] - 2098);
              qs[r * n + col] = (top && rt < ntop) ? xm[rt * n + col] + myw : myw;
            }
          }
        }
      }
    }
    fence_proxy_async_smem();  // the staged rows of Q -> the bulk store
    tc_fence_before();
    __syncthreads();  // tensor memory read before the next chunk's products; Q staged
    tc_fence_after();
    if (tid == 0) {
      const uint32_t bytes = static_cast<uint32_t>(crows) * n * 8;
      const uint32_t bulk = (reinterpret_cast<uintptr_t>(yq) & 15) == 0 ? (bytes & ~15u) : 0u;
      for (uint32_t off = 0; off < bulk; off += kBulkChunk) {
        const uint32_t len = bulk - off < kBulkChunk ? bulk - off : kBulkChunk;
        bulk_s2g(reinterpret_cast<char*>(yq) + off, reinterpret_cast<const char*>(qs) + off, len);
      }
      if (bulk > 0) bulk_commit();
      for (uint32_t e = bulk / 8; e < bytes / 8; ++e) yq[e] = qs[e];  // the unaligned tail
    }
    if (nt < 0) break;
    t = nt;
    c0 = nc0;
    body = body_next;
  }
  // a copy still in flight after an error: wait for it (bounded) before the
  // shared memory is released; the last bulk stores complete
  if (!ok && pend) mbar_wait_bounded(lbar, lph);
  if (tid == 0) bulk_wait_all();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, NC);
}

#endif  // __CUDACC__ && TSQR_OZ_KERNELS

// ---------------------------------------------------------------------------
// The Gram entries v_i^T v_c (i < c) of each tile's Householder vectors, for
// the compact-WY T factors (T_jj = tau_j, T(0:j, j) = -tau_j T(0:j, 0:j)
// G(0:j, j)), on the tensor cores by the same error-free splitting: the
// binary64 Step 1 then leaves these dot products out of its column loop.
//
// Per chunk of up to 128 rows of a tile: column c of V (the chunk's rows of
// Y; tile 0's top rows read as the unit lower Y_top) is written against its
// largest exponent E_c as 64-bit integers cut into S = 8 digits of 8 bits
// (64 bits, not Step 3's 56: a dot product over K rows gathers K digit
// truncations, so K = 128 needs about 7 more bits to stay at the binary64
// level).  The products of V^T V are D_st = Vdigits_s^T Vdigits_t with
// K = 128 rows.  Four digit slices are stacked in the 128 rows of the MMA's M
// dimension (slice j + q in rows 32 q .. 32 q + 31), so one MMA forms the
// products of four A slices with one B slice -- and the B slice is a 32-row
// quarter of the same stacked buffer.  Accumulator region e (32 columns)
// takes the pairs (j, t) with j + t = e for j in {0, 4}, so its quarter q
// holds diagonal d = e + q from at most 2 x 128 products of 8-bit digits:
// integers below 2 x 128 x 255^2 < 2^24, exact in binary32.  The epilogue
// sums P = sum_d D_d 2^(8 (7 - d) - 17) in 64-bit integers per (i, c),
// rounds once to binary64 with the scale 2^(E_i + E_c - 2099), and adds it
// to the tile's Gram in binary64 (a few chunks per tile).  The diagonals
// d >= 8 and the digit truncation weigh about 2^-54 of the column scales.
// ---------------------------------------------------------------------------
constexpr int kGmThreads = 256;
constexpr int kGmK = 128;       // rows per chunk = the MMA's K
constexpr int kGmDigits = 8;
constexpr int kGmBits = 8;
constexpr int kGmMaxN = 32;     // one 32-row quarter per digit slice
constexpr int kGmShift = 17;    // P = sum_d D_d 2^(8 (7-d) - kGmShift) fits 63 bits
constexpr int kGmRegions = 8;   // accumulator regions e = j + t <= 7
constexpr int kGmTmemCols = 256;
constexpr int kGmPart = 33;     // row stride of the epilogue's partial sums (8-byte words)
constexpr int kGmEntries = (kGmMaxN * kGmMaxN + kGmThreads - 1) / kGmThreads;  // Gram entries per thread

static_assert(4 * 32 * kGmPart * 8 <= 2 * 128 * kGmK * 2, "the partial sums fit the two digit buffers");
struct GramOzSmem {
  size_t ys, p0, p4, red, cexp, gacc, bar, lbar, tslot, total;
  TSQR_HD GramOzSmem(int n) {
    size_t o = 0;
    ys = o; o = align_up(o + (size_t)kGmK * n * 8, 128);       // the chunk's rows of Y
    p0 = o; o = align_up(o + 128 * kGmK * 2, 128);            // digit slices 0..3 stacked (binary16)
    p4 = o; o = align_up(o + 128 * kGmK * 2, 128);            // digit slices 4..7 stacked
    red = o; o = align_up(o + 8 * 32 * 4, 16);                // column exponents per warp
    cexp = o; o = align_up(o + 32 * 4, 16);                   // column exponents of the chunk
    gacc = o; o = align_up(o + (size_t)n * n * 8, 16);        // the tile's Gram (binary64)
    bar = o; o = align_up(o + 8, 8);
    lbar = o; o = align_up(o + 8, 8);
    tslot = o; o = align_up(o + 8, 16);
    total = o;
  }
};

#if defined(__CUDACC__) && defined(TSQR_OZ_KERNELS)

// P 2^s as binary64 for a nonzero 64-bit integer P (see oz_neg_scaled).
__device__ __forceinline__ double oz_scaled(long long P, int s) { return oz_neg_scaled(-P, s); }

// Y:   m x n binary64 (Householder vectors as Step 1 wrote them; tile 0's
//      rows < n hold R on and above the diagonal, read as the unit lower Y_top).
// Tst: kt slots of n x n binary64 per block; the Gram entries G(i, c), i < c,
//      go to the slot's strictly upper triangle (tau, on the diagonal, is
//      Step 1's).
// Launch: gridDim = p, blockDim = kGmThreads, dynamic smem = GramOzSmem(n).
__global__ void __launch_bounds__(kGmThreads, 2)
    k_gram_oz(const double* __restrict__ Yg, int64_t m, int n, int b, int B, int bt, int kt, double* Tst,
              int32_t* status) {
  constexpr uint32_t kLbo = 128, kSbo = (kGmK / 8) * 128;   // 2,048: next 8-row group
  constexpr uint32_t kQuarter = 4 * kSbo;                     // 32 rows = one digit slice
  extern __shared__ __align__(1024) unsigned char smem[];
  const GramOzSmem L(n);
  double* ys = reinterpret_cast<double*>(smem + L.ys);
  char* pdig[2] = {reinterpret_cast<char*>(smem + L.p0), reinterpret_cast<char*>(smem + L.p4)};
  int* red = reinterpret_cast<int*>(smem + L.red);
  int* cexp = reinterpret_cast<int*>(smem + L.cexp);
  double* gacc = reinterpret_cast<double*>(smem + L.gacc);
  // epilogue: 4 x 32 x 32 partial sums at row stride kGmPart (odd in 8-byte
  // words: a warp's 32 rows, and a row's 32 columns, fall in distinct banks);
  // 33.8 KB over the two digit buffers (adjacent), free once the products
  // completed
  long long* part = reinterpret_cast<long long*>(smem + L.p0);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
  uint64_t* lbar = reinterpret_cast<uint64_t*>(smem + L.lbar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.tslot);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nn = n * n;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * b;
  const int rows = static_cast<int>(m - row0 < b ? m - row0 : b);
  const int ntiles = rows <= B ? 1 : 1 + (rows - B + bt - 1) / bt;
  const int ntop = rows < n ? rows : n;
  const uint32_t idesc = tc_idesc_f16(128, 32);

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(lbar, 1);
    fence_mbar_init();
  }
  if (warp == 0) tc_alloc(tslot, kGmTmemCols);
  for (int idx = tid; idx < nn; idx += kGmThreads) gacc[idx] = 0.0;
  // this thread's entries of the n x n Gram: pr = tid + e kGmThreads = i n + c
  // (past n x n: i = c = 0, never an entry above the diagonal)
  int ei[kGmEntries], ec[kGmEntries];
#pragma unroll
  for (int e = 0; e < kGmEntries; ++e) {
    const int pr = tid + e * kGmThreads;
    ei[e] = pr < nn ? pr / n : 0;
    ec[e] = pr < nn ? pr - (pr / n) * n : 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  auto tile_rows = [&](int t, int& tr0, int& cnt) {
    tr0 = t == 0 ? 0 : B + (t - 1) * bt;
    cnt = t == 0 ? (rows < B ? rows : B) : (rows - tr0 < bt ? rows - tr0 : bt);
  };
  auto issue = [&](int t, int c0) {
    int tr0, cnt;
    tile_rows(t, tr0, cnt);
    const int crows = cnt - c0 < kGmK ? cnt - c0 : kGmK;
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
  bool pend = false, ok = true;
  int t = 0, c0 = 0;
  uint32_t body = issue(t, c0);
  pend = body > 0;
  for (;;) {
    int tr0, cnt;
    tile_rows(t, tr0, cnt);
    const int crows = cnt - c0 < kGmK ? cnt - c0 : kGmK;
    const double* yq = Yg + (row0 + tr0 + c0) * n;
    const bool top = (t == 0);
    if (body > 0) {
      ok = mbar_wait_bounded(lbar, lph);
      if (ok) {
        lph ^= 1u;
        pend = false;
      }
    }
    for (int e = static_cast<int>(body / 8) + tid; e < crows * n; e += kGmThreads) ys[e] = yq[e];
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok) {
      if (tid == 0) set_status(status, TSQR_ERR_TIMEOUT);
      break;
    }
    // the value of entry (r, c) of the chunk's V (tile 0's top rows: unit lower)
    auto vval = [&](int r, int c) -> double {
      if (r >= crows || c >= n) return 0.0;
      if (top && c0 + r < ntop && c >= c0 + r) return c == c0 + r ? 1.0 : 0.0;
      return ys[r * n + c];
    };
    // ---- column exponents: warp w scans rows 16 w .. 16 w + 15, lane = column
    {
      int emax = 1;
      for (int r = 16 * warp; r < 16 * warp + 16; ++r) {
        int e;
        uint64_t mant;
        uint32_t ng;
        oz_unpack(vval(r, lane), e, mant, ng);
        if (mant != 0 && e > emax) emax = e;
      }
      red[warp * 32 + lane] = emax;
      __syncthreads();
      if (tid < 32) {
        int mx = red[tid];
        for (int w = 1; w < 8; ++w) mx = red[w * 32 + tid] > mx ? red[w * 32 + tid] : mx;
        cexp[tid] = mx;
      }
      __syncthreads();
    }
    // ---- digits: thread (column c, rows 8 kg .. 8 kg + 7) writes, for each
    //      slice s, one 16-byte core row of operand row (s % 4) 32 + c of the
    //      stacked buffer s / 4; a quarter-warp covers 8 consecutive columns
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      const int c = (lane & 7) + 8 * (lane >> 3);  // = lane
      const int kg = pass * 8 + warp;
      const int ec = cexp[c];
      uint64_t F[8];
      uint32_t ng[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        int e;
        uint64_t mant;
        oz_unpack(vval(8 * kg + i, c), e, mant, ng[i]);
        const int sh = ec - e;
        F[i] = sh >= 64 ? 0ull : ((mant << 11) >> sh);  // 64-bit fixed point
      }
      uint32_t sg[4], lo[8], hi[8];
#pragma unroll
      for (int j = 0; j < 4; ++j) sg[j] = (ng[2 * j] << 15) | (ng[2 * j + 1] << 31);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        lo[i] = static_cast<uint32_t>(F[i]);
        hi[i] = static_cast<uint32_t>(F[i] >> 32);
      }
#pragma unroll
      for (int sl = 0; sl < kGmDigits; ++sl) {
        const int byte = kGmDigits - 1 - sl;  // digit sl is byte 7 - sl of F
        const int jb = byte & 3;
        const uint32_t sel = static_cast<uint32_t>(jb | ((4 + jb) << 8));
        uint32_t h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t wa = byte >= 4 ? hi[2 * j] : lo[2 * j];
          const uint32_t wb = byte >= 4 ? hi[2 * j + 1] : lo[2 * j + 1];
          const uint32_t biased = (__byte_perm(wa, wb, sel) & 0x00FF00FFu) | 0x64006400u;
          uint32_t d;
          asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(biased), "r"(0x64006400u));
          h[j] = d ^ sg[j];
        }
        const int row = (sl & 3) * 32 + c;  // operand row in the stacked buffer
        *reinterpret_cast<uint4*>(pdig[sl >> 2] + ((row / 8) * (kGmK / 8) + kg) * 128 + (row % 8) * 16) =
            make_uint4(h[0], h[1], h[2], h[3]);
      }
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // ---- prefetch the next chunk (tiles first to last)
    int nt = t, nc0 = c0 + kGmK;
    if (nc0 >= cnt) {
      nt = t + 1;
      nc0 = 0;
    }
    const uint32_t body_next = nt < ntiles ? issue(nt, nc0) : 0u;
    pend = body_next > 0;
    // ---- products: region e = j + t of the stacked buffer j in {0, 4} with
    //      B slice t (a quarter of the stacked buffer t / 4)
    if (tid == 0) {
      // straight-line issue (descriptor = base + byte offset >> 4); the two
      // stacked buffers are adjacent, p4 = p0 + 32 KB
      const uint64_t d0 = tc_smem_desc(smem_u32(pdig[0]), kLbo, kSbo);
      constexpr uint32_t kBuf = 128 * kGmK * 2;
#pragma unroll
      for (int e = 0; e < kGmRegions; ++e) {
#pragma unroll
        for (int j = 0; j <= 4 && j <= e; j += 4) {
          const int tb = e - j;  // B slice
          const uint32_t aoff = j == 0 ? 0u : kBuf;
          const uint32_t boff = (tb < 4 ? 0u : kBuf) + static_cast<uint32_t>(tb & 3) * kQuarter;
#pragma unroll
          for (int kb = 0; kb < kGmK / 16; ++kb)
            tc_mma_f16(tmem + static_cast<uint32_t>(e * 32), d0 + ((aoff + kb * 256) >> 4),
                       d0 + ((boff + kb * 256) >> 4), idesc, (j > 0 || kb > 0) ? 1 : 0);
        }
      }
      tc_commit(bar);
    }
    ok = __syncthreads_and(mbar_wait_bounded(bar, parity) ? 1 : 0) != 0;
    parity ^= 1u;
    tc_fence_after();
    if (!ok) {
      if (tid == 0) set_status(status, TSQR_ERR_TIMEOUT);
      break;
    }
    // ---- epilogue: warp w reads lane quarter q = w % 4 (row i = lane of
    //      diagonal offset q) and columns 16 (w / 4) .. + 15 of each region
    //      e <= 7 - q, and sums its share of P into part[q][i][c]
    {
      const int q = warp & 3, cb = 16 * (warp >> 2);
      long long acc[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[i] = 0;
#pragma unroll 1
      for (int e = 0; e + q < kGmDigits; ++e) {
        uint32_t v[8], w2[8];
        const uint32_t ta = tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(e * 32 + cb);
        tc_ld_x8(ta, v);
        tc_ld_x8(ta + 8, w2);
        tc_wait_ld();
        const int sh = kGmBits * (kGmDigits - 1 - (e + q)) - kGmShift;
        if (sh >= 0) {  // warp-uniform: one shift direction per region
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            acc[i] += static_cast<long long>(__float2int_rz(__uint_as_float(v[i]))) << sh;
            acc[8 + i] += static_cast<long long>(__float2int_rz(__uint_as_float(w2[i]))) << sh;
          }
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            acc[i] += static_cast<long long>(__float2int_rz(__uint_as_float(v[i]))) >> -sh;
            acc[8 + i] += static_cast<long long>(__float2int_rz(__uint_as_float(w2[i]))) >> -sh;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) part[(q * 32 + lane) * kGmPart + cb + i] = acc[i];
    }
    tc_fence_before();
    __syncthreads();  // partial sums complete; tensor memory read
    tc_fence_after();
#pragma unroll
    for (int e = 0; e < kGmEntries; ++e) {
      const int pr = tid + e * kGmThreads, i = ei[e], c = ec[e];
      if (c > i) {  // entries past n x n have c = i = 0
        const long long P = part[i * kGmPart + c] + part[(32 + i) * kGmPart + c] +
                            part[(64 + i) * kGmPart + c] + part[(96 + i) * kGmPart + c];
        if (P != 0) gacc[pr] += oz_scaled(P, cexp[i] + cexp[c] - 2099);
      }
    }
    const bool last_of_tile = nc0 == 0;  // the next chunk starts a new tile (or none is left)
    if (last_of_tile) {
      __syncthreads();
      double* Tout = Tst + (static_cast<int64_t>(blockIdx.x) * kt + t) * nn;
#pragma unroll
      for (int e = 0; e < kGmEntries; ++e) {
        const int pr = tid + e * kGmThreads;
        if (pr < nn) {
          if (ec[e] > ei[e]) Tout[pr] = gacc[pr];
          gacc[pr] = 0.0;
        }
      }
    }
    __syncthreads();  // part (over the digit buffer) and gacc are free again
    if (nt >= ntiles) break;
    t = nt;
    c0 = nc0;
    body = body_next;
  }
  if (!ok && pend) mbar_wait_bounded(lbar, lph);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, kGmTmemCols);
}

#endif  // __CUDACC__ && TSQR_OZ_KERNELS


}  // namespace tsqr
