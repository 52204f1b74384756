// tc_kernels.cuh -- Step 3 (Sec. III-B) for binary32 data with the product
// Y_i W_i on the 5th-generation tensor cores: tcgen05.mma kind::tf32, the
// accumulator in tensor memory.  3xTF32 split precision: Y = Yh + Yl and
// W = Wh + Wl with Yh, Yl, Wh, Wl rounded to TF32, Y W ~ Yh Wh + Yh Wl + Yl Wh
// (the dropped Yl Wl is below binary32 rounding).
//
// n <= kTcMaxN, two launches.  A row block's Q is H_0 H_1 .. H_{k-1} [C; 0],
// H_t = I - Y_t T_t Y_t^T the compact-WY factor of its tile t.  Applied last
// to first, every tile t > 0 meets the running coefficient X only in its
// carried triangle (Y_t = [I; V_t] there), so its W_t = T_t X and the update
// X -= W_t involve n x n matrices alone; tile 0 adds Y_top^T.  k_w_chain runs
// that chain per block on the CUDA cores and leaves -W_t, split into TF32
// hi and lo parts, in T slot t and X_0 in the block's C.  Every 128-row
// chunk of every tile is then an independent product Q = Y (-W_t) (+ X_0 on
// the block's first n rows), which k_form_q_tc streams: a persistent CTA per
// SM takes a contiguous run of chunks; two groups of four warps take
// alternate chunks, so one group's TF32 split and write-back overlap the
// other's MMA.  A thread owns one row of a chunk (its tensor-memory lane): it
// splits the row staged by the bulk copy into A_hi / A_lo columns of tensor
// memory (tcgen05.st), and after the MMA chain reads its row of the
// accumulator back (tcgen05.ld) into the same staging row, which one bulk
// copy then writes over Y.
//
// The wide form (n > kTcMaxN, k_form_q_tcw) keeps one CTA per block, forms W
// per tile on the CUDA cores and stages A in shared memory.
//
// B operand layout (shared memory): no swizzle, K-major: core matrices of 8
// rows x 16 bytes (4 TF32 values); element (c, k) at ((c/8) * K/4 + k/4) *
// 128 + (c%8) * 16 + (k%4) * 4 bytes, so the descriptor's leading-dimension
// offset (next core along K) is 128 bytes and its stride offset (next 8-row
// group) K/4 * 128.
#pragma once

#include <cstdint>

#include "device.cuh"
#include "layout.cuh"
#include "chunks.cuh"
#include "tcgen05.cuh"

namespace tsqr {

constexpr int kTcM = kChunkM;    // rows per MMA chunk (TMEM lanes)
constexpr int kTcThreads = 512;  // the wide form: 16 warps, warp w reads TMEM lanes 32 (w % 4) ..
constexpr int kTcMaxN = 64;      // largest n of the streaming form

TSQR_HD constexpr int tc_k(int n) { return (n + 7) / 8 * 8; }     // K: MMA K step is 8
TSQR_HD constexpr int tc_n(int n) { return (n + 15) / 16 * 16; }  // N: multiple of 16 at M = 128
TSQR_HD constexpr int tc_cols(int n) { return tc_n(n) <= 32 ? 32 : (tc_n(n) <= 64 ? 64 : 128); }  // TMEM alloc

// ---- the streaming form (n <= kTcMaxN)
constexpr int kTqGroupWarps = 8;                          // a row group: 2 warps per 32-row lane quarter
constexpr int kTqGroupThreads = 32 * kTqGroupWarps;
constexpr int kTqBuildWarps = 2;                         // B operand builders
constexpr int kTqThreads = (2 * kTqGroupWarps + 2 + kTqBuildWarps) * 32;  // row groups, MMA, copy, builders
constexpr int kWcThreads = 256;  // k_w_chain
constexpr int kWcMaxE = (kTcMaxN * kTcMaxN + kWcThreads - 1) / kWcThreads;  // T entries per thread
constexpr int kTqMinSmem = 120 * 1024;  // one CTA per SM (tensor memory is sized for one)
// tensor-memory columns of one group: A_hi (K), A_lo (K), D (N), as a power of two
TSQR_HD constexpr int tq_gcols(int n) {
  return 2 * tc_k(n) + tc_n(n) <= 32 ? 32
       : (2 * tc_k(n) + tc_n(n) <= 64 ? 64 : (2 * tc_k(n) + tc_n(n) <= 128 ? 128 : 256));
}

// Shared memory of k_form_q_tc: 2 nb Y buffers (a chunk as one contiguous
// copy, row stride n, after a head offset below 16 bytes; for n % 8 == 0 as
// 16-row groups 16 bytes apart, see tq_sidx), the B operands of
// two tiles (by ordinal parity), the mbarriers (full[6], aready[2], dfull[2],
// qstaged[6], bready[2], bfree[2]) and the chunk descriptors (one per Y
// buffer, 48 bytes each).
struct FormQTcSmem {
  size_t ybuf, ybytes, bop, bbytes, bars, desc, tslot, total;
  int nb;  // Y buffers per group (3 where they fit, else 2)
  TSQR_HD FormQTcSmem(int n) {
    const size_t K = tc_k(n), N = tc_n(n);
    ybytes = align_up((size_t)kTcM * n * 4 + 128, 128);  // + a head offset or the 16-row groups' stagger
    bbytes = 2 * N * K * 4;  // hi, then lo
    nb = 6 * ybytes + 2 * bbytes + 1536 <= 232448 ? 3 : 2;
    size_t o = 0;
    ybuf = o; o += 2 * (size_t)nb * ybytes;
    bop = o; o = align_up(o + 2 * bbytes, 128);
    bars = o; o += 20 * 8;
    desc = o; o += 6 * 48;
    tslot = o; o = align_up(o + 8, 16);
    total = o;
  }
};

// k_w_chain: T_t^T, X and Z (binary32, n x n each at row stride n rounded up
// to 4, contiguous)
TSQR_HD constexpr int wc_stride(int n) { return (n + 3) / 4 * 4; }
struct WChainSmem {
  size_t ts, xs, zs, total;
  TSQR_HD WChainSmem(int n) {
    const size_t sz = (size_t)n * wc_stride(n) * 4;  // a multiple of 16
    ts = 0;
    xs = sz;
    zs = 2 * sz;
    total = 3 * sz;
  }
};

// The wide form, 64 < n <= TSQR_NMAX: the A operands of a chunk are formed
// and multiplied in up to three K parts (so that X stays in shared memory
// beside one Y buffer and the whole B operand), the next chunk's copy starts
// once the chunk's last A part is formed, the prologue stages T (transposed)
// in the B region and Z / W in the A region, and the epilogue writes Q from
// the tensor-memory loads to global memory directly.
constexpr int kTcwMaxN = 100;
constexpr int kTcwRB = 4, kTcwCB = 5;  // W = T X: a 4 x 5 register block per thread
constexpr int kTcwMaxE = (kTcwMaxN * kTcwMaxN + kTcThreads - 1) / kTcThreads;  // staged entries per thread
TSQR_HD constexpr int tcw_kp(int n) { return ((tc_k(n) + 2) / 3 + 7) / 8 * 8; }  // K per part (multiple of 8)

struct FormQTcwSmem {
  size_t ys, xs, a_hi, a_lo, b_hi, b_lo, bar, lbar, tslot, total;
  TSQR_HD FormQTcwSmem(int n) {
    const size_t K = tc_k(n), N = tc_n(n), KP = tcw_kp(n);
    size_t o = 0;
    ys = o; o = align_up(o + (size_t)kTcM * n * 4, 128);
    xs = o; o = align_up(o + (size_t)n * n * 4, 128);
    a_hi = o; o = align_up(o + kTcM * KP * 4, 128);
    // the A region also holds Z / W (n x n) during a tile's prologue
    const size_t ap = kTcM * KP * 4, nn4 = (size_t)n * n * 4;
    a_lo = o; o = align_up(o + (nn4 > 2 * ap ? nn4 - ap : ap), 128);
    b_hi = o; o = align_up(o + N * K * 4, 128);
    b_lo = o; o = align_up(o + N * K * 4, 128);
    bar = o; o = align_up(o + 8, 8);
    lbar = o; o = align_up(o + 8, 8);
    tslot = o; o = align_up(o + 8, 16);
    total = o;
  }
};

// The device code is compiled only in the translation unit that launches it
// (kern_tc.cu); the planner includes this header for the geometry above.
#if defined(__CUDACC__) && defined(TSQR_TC_KERNELS)

// x rounded to TF32 (10 fraction bits), to nearest with ties away from
// zero: half of the dropped 13 bits' weight is added to the magnitude bits,
// which are then cut (finite x, two integer operations).
__device__ __forceinline__ float tf32_round(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}

// The W chain of Step 3 for one row block per CTA (binary32, CUDA cores):
//   X = C;  for t = k-1 .. 1: W_t = T_t X, X -= W_t;  W_0 = T_0 (Y_top^T X)
// with Y_top the block's first min(rows, n) rows of Y (unit lower
// triangular).  Writes -W_t split into TF32 parts, hi then lo (n x n each,
// row-major, binary32), over T slot t, and X_0 = X (binary32) over the first
// half of the block's C; T_t and C are read before they are written.
// W = T src runs as 4 x 4 register blocks (rows kk0 .., columns c0 ..) read
// with 16-byte shared loads: T is staged transposed and every n x n operand
// at row stride np = n rounded up to 4, the padding zero.
// Launch: gridDim = p, blockDim = kWcThreads, dynamic smem = WChainSmem(n).
__global__ void __launch_bounds__(kWcThreads, 3)
    k_w_chain(const float* __restrict__ Yg, int64_t m, int n, int64_t b, int B, int bt, int kt, double* Tg,
              double* Cg, int64_t cblocks) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const WChainSmem L(n);
  float* ts = reinterpret_cast<float*>(smem + L.ts);
  float* xs = reinterpret_cast<float*>(smem + L.xs);
  float* zs = reinterpret_cast<float*>(smem + L.zs);
  const int tid = threadIdx.x, nn = n * n, np = wc_stride(n), nq = np / 4;
  const int64_t blk = blockIdx.x, row0 = blk * b;
  const int rows = static_cast<int>(m - row0 < b ? m - row0 : b);
  const int ntiles = rows <= B ? 1 : 1 + (rows - B + bt - 1) / bt;
  const int ntop = rows < n ? rows : n;
  const int64_t cb = cblocks == 1 ? 0 : blk;
  for (int idx = tid; idx < 3 * n * np; idx += kWcThreads) ts[idx] = 0.0f;  // ts, xs, zs and their padding
  __syncthreads();
  for (int idx = tid; idx < nn; idx += kWcThreads) xs[(idx / n) * np + idx % n] = static_cast<float>(Cg[cb * nn + idx]);
  const bool wblk = tid < nq * nq;
  const int kk0 = (tid / nq) * 4, c0 = (tid % nq) * 4;
  double tp[kWcMaxE];  // T of the next tile, fetched one step ahead
  auto fetch_t = [&](int t) {
    const double* Tb = Tg + (blk * kt + t) * nn;
#pragma unroll
    for (int e = 0; e < kWcMaxE; ++e) {
      const int idx = tid + e * kWcThreads;
      tp[e] = idx < nn ? Tb[idx] : 0.0;
    }
  };
  fetch_t(ntiles - 1);
  for (int t = ntiles - 1; t >= 0; --t) {
    const float* src = xs;
    if (t == 0) {
      // Z = Y_top^T X: Z[kk] = X[kk] + sum_{kk < r < ntop} Y[r][kk] X[r] (zero for kk >= ntop)
      for (int idx = tid; idx < ntop * n; idx += kWcThreads) ts[(idx / n) * np + idx % n] = Yg[row0 * n + idx];
      __syncthreads();
      if (wblk) {
        float zb[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float4 x = *reinterpret_cast<const float4*>(xs + (kk0 + r < n ? kk0 + r : 0) * np + c0);
          const bool in = kk0 + r < ntop;
          zb[r][0] = in ? x.x : 0.0f;
          zb[r][1] = in ? x.y : 0.0f;
          zb[r][2] = in ? x.z : 0.0f;
          zb[r][3] = in ? x.w : 0.0f;
        }
        for (int i = kk0 + 1; i < ntop; ++i) {
          const float4 y4 = *reinterpret_cast<const float4*>(ts + i * np + kk0);
          const float4 x4 = *reinterpret_cast<const float4*>(xs + i * np + c0);
          const float yv[4] = {i > kk0 ? y4.x : 0.0f, i > kk0 + 1 ? y4.y : 0.0f, i > kk0 + 2 ? y4.z : 0.0f,
                               i > kk0 + 3 ? y4.w : 0.0f};
          const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) zb[r][c] = fmaf(yv[r], xv[c], zb[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (kk0 + r < n)
            *reinterpret_cast<float4*>(zs + (kk0 + r) * np + c0) = make_float4(zb[r][0], zb[r][1], zb[r][2], zb[r][3]);
      }
      __syncthreads();  // Y_top's reads of ts are done before T_0 is staged
      src = zs;
    }
    // T_t transposed into ts (upper triangle; binary64 rounded to binary32)
#pragma unroll
    for (int e = 0; e < kWcMaxE; ++e) {
      const int idx = tid + e * kWcThreads;
      if (idx < nn) {
        const int kk = idx / n, i = idx - kk * n;
        ts[i * np + kk] = i >= kk ? static_cast<float>(tp[e]) : 0.0f;
      }
    }
    if (t > 0) fetch_t(t - 1);
    __syncthreads();
    float wb[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) wb[r][c] = 0.0f;
    if (wblk) {
      for (int i = kk0; i < n; ++i) {
        const float4 t4 = *reinterpret_cast<const float4*>(ts + i * np + kk0);
        const float4 s4 = *reinterpret_cast<const float4*>(src + i * np + c0);
        const float tv[4] = {t4.x, t4.y, t4.z, t4.w}, sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) wb[r][c] = fmaf(tv[r], sv[c], wb[r][c]);
      }
    }
    __syncthreads();  // every read of ts and src is done
    float* Wout = reinterpret_cast<float*>(Tg + (blk * kt + t) * nn);
    if (t == 0) {
      float* X0 = reinterpret_cast<float*>(Cg + cb * nn);  // C was read into xs
      for (int idx = tid; idx < nn; idx += kWcThreads) X0[idx] = xs[(idx / n) * np + idx % n];
    }
    if (wblk) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int kk = kk0 + r, cc = c0 + c;
          if (kk < n && cc < n) {
            const float hv = tf32_round(-wb[r][c]);
            Wout[kk * n + cc] = hv;
            Wout[nn + kk * n + cc] = tf32_round(-wb[r][c] - hv);
            if (t > 0) xs[kk * np + cc] -= wb[r][c];
          }
        }
    }
    __syncthreads();
  }
}

// What the copy warp tells the row groups and the MMA thread about the chunk
// in a Y buffer.  The chunk's elements [0, crows n) outside its
// 16-byte-aligned body are [0, nh) and [t0, crows n); its first element sits
// at float hoff of the buffer.
struct TqDesc {
  int64_t off;   // element offset of the chunk in Y
  int64_t slot;  // T slot of its tile
  int64_t blk;   // its block
  int hoff, nh, t0, crows, ntop, pad;
};

// Float offset of row r of a staged chunk: row-major at stride n, or (STAG,
// n % 8 == 0) in 16-row groups each 16 bytes further on, so that rows
// 16 apart start 4 banks apart.
template <bool STAG>
__device__ __forceinline__ int tq_sidx(int r, int n) {
  return STAG ? (r >> 4) * (16 * n + 4) + (r & 15) * n : r * n;
}

// 8 values of a staged row from column k0 (k0 + 8 <= n), VW-wide shared loads.
template <int VW>
__device__ __forceinline__ void tq_ld8(const float* p, float (&y)[8]) {
  if constexpr (VW == 4) {
    const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
    y[0] = a.x; y[1] = a.y; y[2] = a.z; y[3] = a.w; y[4] = b.x; y[5] = b.y; y[6] = b.z; y[7] = b.w;
  } else if constexpr (VW == 2) {
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      const float2 a = *reinterpret_cast<const float2*>(p + i);
      y[i] = a.x;
      y[i + 1] = a.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) y[i] = p[i];
  }
}
template <int VW>
__device__ __forceinline__ void tq_st8(float* p, const float (&x)[8]) {
  if constexpr (VW == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
    *reinterpret_cast<float4*>(p + 4) = make_float4(x[4], x[5], x[6], x[7]);
  } else if constexpr (VW == 2) {
#pragma unroll
    for (int i = 0; i < 8; i += 2) *reinterpret_cast<float2*>(p + i) = make_float2(x[i], x[i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) p[i] = x[i];
  }
}

// The TF32 split of one thread's staged row `ys` (valid: rv) into tensor
// memory: its half h of the 8-column pieces (at most four, K <= 64), A_hi at
// column k0, A_lo at K + k0; columns n .. K-1 are zero.
template <int VW>
__device__ __forceinline__ void tq_split(const float* ys, bool rv, int n, int K, int h, uint32_t tl) {
  float y[4][8];  // all pieces first, so the shared loads overlap
#pragma unroll
  for (int pc = 0; pc < 4; ++pc) {
    const int k0 = 8 * (h + 2 * pc);
    if (k0 < K) {
      if (rv && k0 + 8 <= n) {
        tq_ld8<VW>(ys + k0, y[pc]);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) y[pc][i] = (rv && k0 + i < n) ? ys[k0 + i] : 0.0f;
      }
    }
  }
#pragma unroll
  for (int pc = 0; pc < 4; ++pc) {
    const int k0 = 8 * (h + 2 * pc);
    if (k0 < K) {
      uint32_t hv[8], lv[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float hf = tf32_round(y[pc][i]);
        hv[i] = __float_as_uint(hf);
        lv[i] = __float_as_uint(tf32_round(y[pc][i] - hf));
      }
      tc_st_x8(tl + static_cast<uint32_t>(k0), hv);
      tc_st_x8(tl + static_cast<uint32_t>(K + k0), lv);
    }
  }
}

// Q of one thread's row, its half h of the 8-column pieces of the
// accumulator (tensor-memory columns 2K ..), into its staging row yw.
template <int VW>
__device__ __forceinline__ void tq_epi(float* yw, bool rv, int n, int K, int h, uint32_t tl) {
  uint32_t v[4][8];
#pragma unroll
  for (int pc = 0; pc < 4; ++pc) {
    const int c0 = 8 * (h + 2 * pc);
    if (c0 < n) tc_ld_x8(tl + static_cast<uint32_t>(2 * K + c0), v[pc]);
  }
  tc_wait_ld();
  if (!rv) return;
#pragma unroll
  for (int pc = 0; pc < 4; ++pc) {
    const int c0 = 8 * (h + 2 * pc);
    if (c0 < n) {
      float x[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = __uint_as_float(v[pc][i]);
      if (c0 + 8 <= n) {
        tq_st8<VW>(yw + c0, x);
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (c0 + i < n) yw[c0 + i] = x[i];
      }
    }
  }
}

// Step 3, binary32 data, n <= kTcMaxN: Q = Y (-W_t) (+ X_0), the chunks of
// all blocks streamed by a persistent grid (see the file comment).
//   Yg : m x n (binary32), Y as written by k_local_qr; Q is written over it.
//   Tg : the T slots after k_w_chain (-W_t as TF32 hi and lo parts).
//   Cg : the blocks' C after k_w_chain (X_0 in binary32).
// Warp roles:
//   0-7, 8-15  the two row groups (warp w of a group: TMEM lanes 32 (w % 4)
//              .., half w / 4 of the 8-column pieces): TF32 split of the
//              staged rows into tensor memory, then Q from the accumulator;
//   16         lane 0 issues the MMA chains;
//   17         lane 0 issues the bulk copies in and out and describes each
//              chunk in desc[s];
//   18-19      build the B operands of the CTA's tiles in turn (two buffers,
//              by the tile's ordinal in the CTA's run), by cp.async.
// Hand-offs are mbarriers: full[s] (copy into Y buffer s landed, desc[s]
// written), aready[g] (group g's A operands are in tensor memory), dfull[g]
// (its MMA chain completed), qstaged[s] (the Q rows in Y buffer s are staged
// for the copy out), bready[x] / bfree[x] (B buffer x built / no longer
// read).  Chunk i of a CTA's run goes to group i % 2 and Y buffer i % (2 nb).
// No waiter may fall two phases behind a barrier (the parity would alias):
// every barrier's next phase needs a step its waiter takes after observing
// the current one -- which is why qstaged is per buffer (a group reaches its
// next use of buffer s only after the copy out of s, which follows the wait),
// not per group (a group can stage two chunks before the copy thread looks).
// Launch: gridDim <= the SM count, blockDim = kTqThreads, dynamic smem =
// max(FormQTcSmem(n).total, kTqMinSmem).
template <int VW, bool STAG>
__global__ void __launch_bounds__(kTqThreads, 1)
    k_form_q_tc(float* Yg, int64_t m, int n, int64_t b, int B, int bt, int kt, int64_t p,
                const double* __restrict__ Tg, const double* __restrict__ Cg, int32_t* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const FormQTcSmem L(n);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = tc_k(n), N = tc_n(n), KQ = K / 4, nn = n * n, nbuf = 2 * L.nb;
  const int GC = tq_gcols(n);
  float* ybase = reinterpret_cast<float*>(smem + L.ybuf);
  const int ystride = static_cast<int>(L.ybytes / 4);  // floats per Y buffer
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L.bars);
  uint64_t* aready = full + 6;
  uint64_t* dfull = full + 8;
  uint64_t* qstaged = full + 10;  // one per Y buffer (see below)
  uint64_t* bready = full + 16;
  uint64_t* bfree = full + 18;
  TqDesc* desc = reinterpret_cast<TqDesc*>(smem + L.desc);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.tslot);
  const uintptr_t yaddr = reinterpret_cast<uintptr_t>(Yg);  // VW: the widest row vector Y's alignment allows

  const TqGeom G(m, n, b, B, bt, p);
  const int64_t total = G.total();
  const int64_t lo = total * blockIdx.x / gridDim.x, hi = total * (blockIdx.x + 1) / gridDim.x;
  const int nloc = static_cast<int>(hi - lo);  // chunks of this CTA (a few thousand at most)

  if (tid == 0) {
    for (int s = 0; s < nbuf; ++s) {
      mbar_init(full + s, 1);
      mbar_init(qstaged + s, kTqGroupWarps);
    }
    for (int g = 0; g < 2; ++g) {
      mbar_init(aready + g, kTqGroupWarps);
      mbar_init(dfull + g, 1);
      mbar_init(bready + g, 1);
      mbar_init(bfree + g, 1);
    }
    fence_mbar_init();
  }
  if (warp == 0) tc_alloc(tslot, static_cast<uint32_t>(2 * GC));
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  bool ok = true;

  if (warp < 2 * kTqGroupWarps) {
    // ================= a row group =================
    const int g = warp / kTqGroupWarps, gw = warp % kTqGroupWarps, q = gw & 3, h = gw >> 2;
    const int gt = tid % kTqGroupThreads;  // thread within the group
    // my row of the chunk: tensor-memory lane L = 32 q + lane holds row L, or
    // with the staggered staging row 16 (L % 8) + L / 8, so that a quarter
    // warp's eight rows lie in eight different 16-row groups
    const int L = 32 * q + lane;
    const int r = STAG ? 16 * (L & 7) + (L >> 3) : L;
    const uint32_t tl = tmem + static_cast<uint32_t>(g * GC) + (static_cast<uint32_t>(32 * q) << 16);
    const int e0 = tq_sidx<STAG>(r, n);  // my row's first element in the staging buffer
    uint32_t fpar = 0, ph = 0;  // Y buffer parities (bit per buffer); the group's barrier parity
    int s = g;
    for (int i = g; i < nloc; i += 2) {
      float* yb = ybase + s * ystride;
      // group-uniform outcomes of the bounded waits (the group meets at named
      // barriers below, so no warp may leave alone)
      if (!named_bar_and(2 + g, kTqGroupThreads, mbar_wait_bounded(full + s, (fpar >> s) & 1u))) {
        ok = false;
        break;
      }
      fpar ^= 1u << s;
      const TqDesc& dc = desc[s];
      const int hoff = dc.hoff, nh = dc.nh, t0 = dc.t0, ntop = dc.ntop, ne = dc.crows * n;
      float* ys = yb + hoff;  // the chunk's staged elements
      const bool rv = r < dc.crows;
      // chunks with unaligned edges or the block's first rows are patched in
      // the staging buffer first (few: a block's first chunk, tile ends)
      const bool plain = ntop == 0 && nh == 0 && t0 == ne;
      if (!plain) {
        const float* yc = Yg + dc.off;
        for (int e = gt; e < nh; e += kTqGroupThreads) ys[e] = yc[e];
        for (int e = t0 + gt; e < ne; e += kTqGroupThreads) ys[e] = yc[e];
        // Y_top is unit lower triangular: its upper part is not Y's
        for (int e = gt; e < ntop * n; e += kTqGroupThreads) {
          const int rr = e / n, k = e - rr * n;
          if (k >= rr) ys[tq_sidx<STAG>(rr, n) + k] = k == rr ? 1.0f : 0.0f;
        }
        named_bar_sync(2 + g, kTqGroupThreads);
      }
      tq_split<VW>(ys + e0, rv, n, K, h, tl);
      tc_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(aready + g);
      // ---- Q rows from the accumulator into the staging rows
      if (!named_bar_and(2 + g, kTqGroupThreads, mbar_wait_bounded(dfull + g, ph))) {
        ok = false;
        break;
      }
      ph ^= 1u;
      tc_fence_after();
      tq_epi<VW>(ys + e0, rv, n, K, h, tl);
      if (!plain) {
        named_bar_sync(2 + g, kTqGroupThreads);
        const float* x0 = reinterpret_cast<const float*>(Cg + dc.blk * nn);
        for (int e = gt; e < ntop * n; e += kTqGroupThreads) {  // Q = [X_0; 0] - Y W
          const int rr = e / n;
          ys[tq_sidx<STAG>(rr, n) + e - rr * n] += x0[e];
        }
        named_bar_sync(2 + g, kTqGroupThreads);
        float* qc = Yg + dc.off;  // the edges go to Y directly (the copy out takes the body)
        for (int e = gt; e < nh; e += kTqGroupThreads) qc[e] = ys[e];
        for (int e = t0 + gt; e < ne; e += kTqGroupThreads) qc[e] = ys[e];
      }
      fence_proxy_async_smem();  // staging rows -> the bulk copy out
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(qstaged + s);
      s += 2;
      if (s >= nbuf) s -= nbuf;
    }
  } else if (warp == 2 * kTqGroupWarps) {
    // ================= the MMA thread =================
    if (lane == 0) {
      const uint32_t idesc = tc_idesc_tf32(kTcM, N);
      const uint32_t lbo = 128, sbo = static_cast<uint32_t>(KQ) * 128;
      const uint32_t b0 = smem_u32(smem + L.bop);
      int64_t cur = -1;
      int tk = -1;  // ordinal of the current tile in this CTA's run
      int s = 0;
      for (int i = 0; i < nloc; ++i) {
        const int g = i & 1;
        if (!mbar_wait_bounded(aready + g, static_cast<uint32_t>(i >> 1) & 1u)) {
          ok = false;
          break;
        }
        const int64_t slot = desc[s].slot;  // written before full[s], which group g waited on
        if (slot != cur) {
          if (tk >= 0) tc_commit(bfree + (tk & 1));  // B buffer of the tile before: free once its chains complete
          ++tk;
          cur = slot;
          if (!mbar_wait_bounded(bready + (tk & 1), static_cast<uint32_t>(tk >> 1) & 1u)) {
            ok = false;
            break;
          }
        }
        tc_fence_after();
        const uint32_t ta = tmem + static_cast<uint32_t>(g * GC);
        const uint32_t d = ta + static_cast<uint32_t>(2 * K);
        const uint32_t bb = b0 + static_cast<uint32_t>(tk & 1) * static_cast<uint32_t>(L.bbytes);
        const uint64_t dbh = tc_smem_desc(bb, lbo, sbo);
        const uint64_t dbl = tc_smem_desc(bb + static_cast<uint32_t>(N * K * 4), lbo, sbo);
        for (int kb = 0; kb < K / 8; ++kb) {
          const uint64_t ko = static_cast<uint64_t>(kb) * 16;  // 256 bytes >> 4
          const uint32_t ah = ta + static_cast<uint32_t>(kb * 8), al = ah + static_cast<uint32_t>(K);
          tc_mma_tf32_ta(d, ah, dbh + ko, idesc, kb > 0);
          tc_mma_tf32_ta(d, ah, dbl + ko, idesc, 1);
          tc_mma_tf32_ta(d, al, dbh + ko, idesc, 1);
        }
        tc_commit(dfull + g);
        if (++s == nbuf) s = 0;
      }
    }
  } else if (warp == 2 * kTqGroupWarps + 1) {
    // ================= the copy thread =================
    if (lane == 0) {
      // describe chunk c (cursor cl) in desc[s] and start its copy in; then
      // copies out in chunk order, each freeing the buffer of the chunk
      // before it for the next copy in
      auto issue = [&](const TqCursor& cl, int s) {
        TqDesc& dd = desc[s];
        const int crows = cl.crows();
        const uintptr_t a = yaddr + static_cast<uintptr_t>(cl.off) * 4;
        const uintptr_t e = a + static_cast<uintptr_t>(crows) * n * 4;
        uintptr_t bs = (a + 15) & ~static_cast<uintptr_t>(15), be = e & ~static_cast<uintptr_t>(15);
        if (be <= bs) be = bs;  // no aligned body
        dd.off = cl.off;
        dd.slot = cl.slot;
        dd.blk = cl.blk;
        dd.hoff = static_cast<int>((a & 15) / 4);
        dd.nh = be > bs ? static_cast<int>((bs - a) / 4) : crows * n;
        dd.t0 = be > bs ? static_cast<int>((be - a) / 4) : crows * n;
        dd.crows = crows;
        dd.ntop = cl.ntop(n);
        const uint32_t body = static_cast<uint32_t>(be - bs);
        mbar_arrive_expect_tx(full + s, body);  // releases desc[s]; body 0: the phase completes now
        if constexpr (STAG) {  // rows 16-byte aligned (no edges): one copy per 16-row group
          float* dst = ybase + s * ystride;
          for (int r0 = 0; r0 < crows; r0 += 16) {
            const int nr = crows - r0 < 16 ? crows - r0 : 16;
            bulk_g2s(dst + tq_sidx<true>(r0, n), Yg + cl.off + static_cast<int64_t>(r0) * n,
                     static_cast<uint32_t>(nr) * n * 4, full + s);
          }
        } else {
          char* dst = reinterpret_cast<char*>(ybase + s * ystride) + (bs - (a & ~static_cast<uintptr_t>(15)));
          for (uint32_t o = 0; o < body; o += kBulkChunk) {
            const uint32_t len = body - o < kBulkChunk ? body - o : kBulkChunk;
            bulk_g2s(dst + o, reinterpret_cast<const char*>(bs) + o, len, full + s);
          }
        }
      };
      uint32_t pend = 0, fpar = 0;  // copies in not yet consumed (bit per buffer); their phase parities
      TqCursor cl;
      if (nloc > 0) cl.set(G, kt, lo);
      int nload = 0, sl = 0;
      for (; nload < nloc && nload < nbuf; ++nload) {
        issue(cl, sl);
        pend |= 1u << sl;
        cl.next(G, kt);
        if (++sl == nbuf) sl = 0;
      }
      int ss = 0;        // buffer of chunk i
      uint32_t qpar = 0;  // qstaged parities, bit per buffer
      for (int i = 0; i < nloc; ++i) {
        if (!mbar_wait_bounded(qstaged + ss, (qpar >> ss) & 1u)) {
          ok = false;
          break;
        }
        qpar ^= 1u << ss;
        // chunk i was consumed (its group staged Q): its copy in completed
        pend &= ~(1u << ss);
        fpar ^= 1u << ss;
        {
          const TqDesc& dd = desc[ss];
          if constexpr (STAG) {
            const float* sp = ybase + ss * ystride;
            for (int r0 = 0; r0 < dd.crows; r0 += 16) {
              const int nr = dd.crows - r0 < 16 ? dd.crows - r0 : 16;
              bulk_s2g(Yg + dd.off + static_cast<int64_t>(r0) * n, sp + tq_sidx<true>(r0, n),
                       static_cast<uint32_t>(nr) * n * 4);
            }
          } else {
            const uintptr_t a = yaddr + static_cast<uintptr_t>(dd.off) * 4;
            const uintptr_t bs = a + static_cast<uintptr_t>(dd.nh) * 4, be = a + static_cast<uintptr_t>(dd.t0) * 4;
            const char* sp =
                reinterpret_cast<const char*>(ybase + ss * ystride) + (bs - (a & ~static_cast<uintptr_t>(15)));
            for (uintptr_t o = 0; o < be - bs; o += kBulkChunk) {
              const uint32_t len = static_cast<uint32_t>(be - bs - o < kBulkChunk ? be - bs - o : kBulkChunk);
              bulk_s2g(reinterpret_cast<char*>(bs) + o, sp + o, len);
            }
          }
          bulk_commit();  // one group per chunk (possibly empty)
        }
        if (i >= 1 && nload < nloc) {
          bulk_wait_read_1();  // chunk i - 1's copy out has read its buffer (sl)
          issue(cl, sl);
          pend |= 1u << sl;
          cl.next(G, kt);
          ++nload;
          if (++sl == nbuf) sl = 0;
        }
        if (++ss == nbuf) ss = 0;
      }
      // copies in flight after an error: wait for them (bounded) before the
      // shared memory is released; the copies out complete in any case
      for (int s = 0; s < nbuf; ++s)
        if (pend & (1u << s)) mbar_wait_bounded(full + s, (fpar >> s) & 1u);
      bulk_wait_all();
    }
  } else {
    // ================= the B builders =================
    // element x of a part (hi or lo) in the core layout: core row it = x / 32,
    // c = (it / KQ) 8 + (x % 32) / 4, k = (it % KQ) 4 + x % 4; builder thread
    // bt takes x = bt + 32 kTqBuildWarps e (so x % 32 is its lane)
    const int btid = tid - (2 * kTqGroupWarps + 2) * 32;
    float* bufs = reinterpret_cast<float*>(smem + L.bop);
    TqCursor ct;  // the CTA's tiles in order: the first chunk's, then one tile on each time
    if (nloc > 0) ct.set(G, kt, lo);
    int64_t last_slot = -1;
    {
      TqCursor ce;  // the tile of the CTA's last chunk
      if (nloc > 0) {
        ce.set(G, kt, hi - 1);
        last_slot = ce.slot;
      }
    }
    const int nx = N * K;
    for (int tk = 0; nloc > 0; ++tk) {
      const int x = tk & 1;
      if (!named_bar_and(1, 32 * kTqBuildWarps,
                         tk < 2 || mbar_wait_bounded(bfree + x, static_cast<uint32_t>((tk - 2) >> 1) & 1u))) {
        ok = false;  // the builders leave together
        break;
      }
      float* bh = bufs + static_cast<size_t>(x) * (L.bbytes / 4);
      float* bl = bh + nx;
      const float* Ws = reinterpret_cast<const float*>(Tg + ct.slot * nn);
      int it = btid >> 5, gc = it / KQ, kq = it % KQ;
      const int cl = lane >> 2, kl = lane & 3;
      for (int xx = btid; xx < nx; xx += 32 * kTqBuildWarps) {
        const int c = gc * 8 + cl, k = kq * 4 + kl;
        if (c < n && k < n) {
          cp_async_4(bh + xx, Ws + k * n + c);
          cp_async_4(bl + xx, Ws + nn + k * n + c);
        } else {
          bh[xx] = 0.0f;
          bl[xx] = 0.0f;
        }
        kq += kTqBuildWarps;  // <= KQ (K >= 8)
        if (kq >= KQ) {
          kq -= KQ;
          ++gc;
        }
      }
      cp_async_wait_all();
      fence_proxy_async_smem();  // generic and cp.async writes -> tensor-core reads
      named_bar_sync(1, 32 * kTqBuildWarps);
      if (btid == 0) mbar_arrive(bready + x);
      if (ct.slot == last_slot) break;
      // one tile on
      ct.c0 = ct.cnt;  // skip to the tile's end, so next() starts the next tile
      ct.off = 0;
      ct.next(G, kt);
    }
  }
  if (!ok) set_status(status, TSQR_ERR_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, static_cast<uint32_t>(2 * GC));
}

// Step 3, binary32 data, tensor-core product, 64 < n <= kTcwMaxN.
//   Yg : m x n (binary32), Y as written by k_local_qr; Q is written over it.
//   Tg : kt slots of n x n binary64 per block (upper triangle).
//   Cg : cblocks blocks of n x n binary64 (cblocks == 1: one C for all).
// Launch: gridDim = p, blockDim = kTcThreads, dynamic smem = FormQTcwSmem(n).
__global__ void __launch_bounds__(kTcThreads, 1)
    k_form_q_tcw(float* Yg, int64_t m, int n, int b, int B, int bt, int kt, const double* __restrict__ Tg,
                 const double* __restrict__ Cg, int64_t cblocks, int32_t* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const FormQTcwSmem L(n);
  float* ys = reinterpret_cast<float*>(smem + L.ys);
  float* xs = reinterpret_cast<float*>(smem + L.xs);
  float* a_hi = reinterpret_cast<float*>(smem + L.a_hi);
  float* a_lo = reinterpret_cast<float*>(smem + L.a_lo);
  float* b_hi = reinterpret_cast<float*>(smem + L.b_hi);
  float* b_lo = reinterpret_cast<float*>(smem + L.b_lo);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
  uint64_t* lbar = reinterpret_cast<uint64_t*>(smem + L.lbar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.tslot);
  float* tts = b_hi;  // prologue: T transposed, tts[i * n + kk] = T[kk][i] (zero below the diagonal)
  float* wst = a_hi;  // prologue: Z (tile 0), then W, row-major n x n

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = tc_k(n), N = tc_n(n), NC = tc_cols(n), KP = tcw_kp(n);
  const int nn = n * n;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * b;
  const int rows = static_cast<int>(m - row0 < b ? m - row0 : b);
  const int ntiles = rows <= B ? 1 : 1 + (rows - B + bt - 1) / bt;
  const int ntop = rows < n ? rows : n;
  const uint32_t idesc = tc_idesc_tf32(kTcM, N);
  const uint32_t lbo = 128;
  const uint32_t sbo_a = static_cast<uint32_t>(KP / 4) * 128, sbo_b = static_cast<uint32_t>(K / 4) * 128;
  const int64_t cb = cblocks == 1 ? 0 : static_cast<int64_t>(blockIdx.x);

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(lbar, 1);
    fence_mbar_init();
  }
  if (warp == 0) tc_alloc(tslot, NC);
  for (int idx = tid; idx < nn; idx += kTcThreads) xs[idx] = static_cast<float>(Cg[cb * nn + idx]);  // X = C
  // this thread's 4 x 5 block of an n x n product: rows kk0 .. kk0 + 3, columns
  // c0b .. c0b + 4; consecutive threads take consecutive column blocks, so a
  // warp spans one or two row blocks and its lanes run (nearly) the same
  // length of the triangular sum
  const int nrb = (n + kTcwRB - 1) / kTcwRB, ncb = (n + kTcwCB - 1) / kTcwCB;
  const bool wblk = tid < nrb * ncb;
  const int kk0 = (tid / ncb) * kTcwRB, c0b = (tid % ncb) * kTcwCB;
  const float inv_n = 1.0f / static_cast<float>(n);
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
    const int crows = cnt - c0 < kTcM ? cnt - c0 : kTcM;
    const float* src = Yg + (row0 + tr0 + c0) * n;
    const uint32_t bytes = static_cast<uint32_t>(crows) * n * 4;
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
  // A operands of the chunk's K columns [k0, k0 + kw) (zero beyond n), split
  // into TF32 hi + lo; warp iteration `it` fills core matrix it (8 rows x 4
  // values) lane by lane; tile 0's top rows are the unit lower Y_top
  auto split_a = [&](int k0, int kw, int crows, bool top, int c0) {
    const int KQ = kw / 4;
    for (int gr = warp; gr < kTcM / 8; gr += kTcThreads / 32) {
      const int r = gr * 8 + (lane >> 2);
      for (int kq = 0; kq < KQ; ++kq) {
        const int it = gr * (KP / 4) + kq, k = k0 + kq * 4 + (lane & 3);
        float y = 0.0f;
        if (r < crows && k < n) {
          y = ys[r * n + k];
          if (top && c0 + r < ntop && k >= c0 + r) y = (k == c0 + r) ? 1.0f : 0.0f;
        }
        const float h = tf32_round(y);
        a_hi[it * 32 + lane] = h;
        a_lo[it * 32 + lane] = tf32_round(y - h);
      }
    }
  };
  auto mma_part = [&](int kb0, int kb1) {
    const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
    for (int kb = kb0; kb < kb1; ++kb) {
      const uint32_t ka = static_cast<uint32_t>(kb - kb0) * 256, kbb = static_cast<uint32_t>(kb) * 256;
      const uint64_t dah = tc_smem_desc(ah + ka, lbo, sbo_a), dal = tc_smem_desc(al + ka, lbo, sbo_a);
      const uint64_t dbh = tc_smem_desc(bh + kbb, lbo, sbo_b), dbl = tc_smem_desc(bl + kbb, lbo, sbo_b);
      tc_mma_tf32(tmem, dah, dbh, idesc, kb > 0 ? 1 : 0);
      tc_mma_tf32(tmem, dah, dbl, idesc, 1);
      tc_mma_tf32(tmem, dal, dbh, idesc, 1);
    }
    tc_commit(bar);
  };

  uint32_t parity = 0, lph = 0;
  bool pend = false, ok = true;
  int t = ntiles - 1, c0 = 0, cur_tile = -1;
  uint32_t body = issue(t, c0);
  pend = body > 0;
  for (;;) {
    int tr0, cnt;
    tile_rows(t, tr0, cnt);
    const int crows = cnt - c0 < kTcM ? cnt - c0 : kTcM;
    float* yq = Yg + (row0 + tr0 + c0) * n;
    const bool top = (t == 0);
    if (body > 0) {
      ok = mbar_wait_bounded(lbar, lph);
      if (ok) {
        lph ^= 1u;
        pend = false;
      }
    }
    for (int e = static_cast<int>(body / 4) + tid; e < crows * n; e += kTcThreads) ys[e] = yq[e];
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok) {
      if (tid == 0) set_status(status, TSQR_ERR_TIMEOUT);
      break;
    }
    if (t != cur_tile) {
      // ---- prologue of tile t: W = T X (tile 0: W = T (Y_top^T X)), X <- X - W, B operands
      cur_tile = t;
      {
        // T, transposed into the B region: all loads in flight before the stores
        const double* Tb = Tg + (static_cast<int64_t>(blockIdx.x) * kt + t) * nn;
        double tv[kTcwMaxE];
#pragma unroll
        for (int e = 0; e < kTcwMaxE; ++e) {
          const int idx = tid + e * kTcThreads;
          tv[e] = idx < nn ? __ldg(Tb + idx) : 0.0;
        }
        // entry idx = kk n + i, kk = floor((idx + 1/2) / n) in binary32 (exact:
        // idx < 10^4 and the quotient lies at least 1/(2n) from an integer)
#pragma unroll
        for (int e = 0; e < kTcwMaxE; ++e) {
          const int idx = tid + e * kTcThreads;
          if (idx < nn) {
            const int kk = __float2int_rz((static_cast<float>(idx) + 0.5f) * inv_n), i = idx - kk * n;
            tts[i * n + kk] = i >= kk ? static_cast<float>(tv[e]) : 0.0f;
          }
        }
      }
      const float* src = xs;
      float w[kTcwRB][kTcwCB];
      if (t == 0) {
        // Z = Y_top^T X, Y_top unit lower triangular (rows < ntop of this chunk, c0 == 0)
#pragma unroll
        for (int r = 0; r < kTcwRB; ++r)
#pragma unroll
          for (int c = 0; c < kTcwCB; ++c) w[r][c] = 0.0f;
        if (wblk) {
#pragma unroll
          for (int r = 0; r < kTcwRB; ++r) {
            const int kk = kk0 + r;
            if (kk < ntop)
#pragma unroll
              for (int c = 0; c < kTcwCB; ++c)
                if (c0b + c < n) w[r][c] = xs[kk * n + c0b + c];
          }
          for (int rr = kk0 + 1; rr < ntop; ++rr) {
            float yv[kTcwRB];
#pragma unroll
            for (int r = 0; r < kTcwRB; ++r) yv[r] = (kk0 + r < rr && kk0 + r < n) ? ys[rr * n + kk0 + r] : 0.0f;
#pragma unroll
            for (int c = 0; c < kTcwCB; ++c) {
              const float xv = c0b + c < n ? xs[rr * n + c0b + c] : 0.0f;
#pragma unroll
              for (int r = 0; r < kTcwRB; ++r) w[r][c] = fmaf(yv[r], xv, w[r][c]);
            }
          }
#pragma unroll
          for (int r = 0; r < kTcwRB; ++r)
#pragma unroll
            for (int c = 0; c < kTcwCB; ++c)
              if (kk0 + r < n && c0b + c < n) wst[(kk0 + r) * n + c0b + c] = w[r][c];
        }
        src = wst;
      }
      __syncthreads();  // T staged (and Z written)
      // W = T src
#pragma unroll
      for (int r = 0; r < kTcwRB; ++r)
#pragma unroll
        for (int c = 0; c < kTcwCB; ++c) w[r][c] = 0.0f;
      if (wblk) {
        for (int i = kk0; i < n; ++i) {
          float tvv[kTcwRB], sv[kTcwCB];
#pragma unroll
          for (int r = 0; r < kTcwRB; ++r) tvv[r] = kk0 + r < n ? tts[i * n + kk0 + r] : 0.0f;
#pragma unroll
          for (int c = 0; c < kTcwCB; ++c) sv[c] = c0b + c < n ? src[i * n + c0b + c] : 0.0f;
#pragma unroll
          for (int r = 0; r < kTcwRB; ++r)
#pragma unroll
            for (int c = 0; c < kTcwCB; ++c) w[r][c] = fmaf(tvv[r], sv[c], w[r][c]);
        }
      }
      __syncthreads();  // every read of the staged T, X and Z is done
      if (wblk) {
#pragma unroll
        for (int r = 0; r < kTcwRB; ++r)
#pragma unroll
          for (int c = 0; c < kTcwCB; ++c) {
            const int kk = kk0 + r, cc = c0b + c;
            if (kk < n && cc < n) {
              wst[kk * n + cc] = w[r][c];
              if (t > 0) xs[kk * n + cc] -= w[r][c];  // coefficient of tile t-1
            }
          }
      }
      __syncthreads();
      // B operands: element (c, k) of B^T = W[k][c], split into TF32 hi + lo
      {
        const int KQ = K / 4;
        for (int gc = warp; gc < N / 8; gc += kTcThreads / 32)
          for (int kq = 0; kq < KQ; ++kq) {
            const int it = gc * KQ + kq;
            const int c = gc * 8 + (lane >> 2), k = kq * 4 + (lane & 3);
            const float x = (c < n && k < n) ? wst[k * n + c] : 0.0f;
            const float h = tf32_round(x);
            b_hi[it * 32 + lane] = h;
            b_lo[it * 32 + lane] = tf32_round(x - h);
          }
      }
      __syncthreads();  // W (in the A region) is read before the A operands overwrite it
    }
    // ---- the K parts: A operands, then their products (the next part's
    //      operands are formed once the previous products have read theirs)
    int nt = t, nc0 = c0 + kTcM;
    if (nc0 >= cnt) {
      nt = t - 1;
      nc0 = 0;
    }
    uint32_t body_next = 0;
    for (int k0 = 0; k0 < K && ok; k0 += KP) {
      const int kw = K - k0 < KP ? K - k0 : KP;
      split_a(k0, kw, crows, top, c0);
      fence_proxy_async_smem();  // A operands -> tensor cores; ys reads -> next bulk copy
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (k0 + kw >= K) {  // ys is free: the next chunk's copy
        body_next = nt >= 0 ? issue(nt, nc0) : 0u;
        pend = body_next > 0;
      }
      if (tid == 0) mma_part(k0 / 8, (k0 + kw) / 8);
      ok = __syncthreads_and(mbar_wait_bounded(bar, parity) ? 1 : 0) != 0;
      parity ^= 1u;
      tc_fence_after();
    }
    if (!ok) {
      if (tid == 0) set_status(status, TSQR_ERR_TIMEOUT);
      break;
    }
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. and the h = w / 4
    //      th group of cw columns; each lane writes its row's 8 columns
    {
      const int q = warp & 3, h = warp >> 2;
      const int cw = ((N / 4 + 7) / 8) * 8;
      const int cend = (h + 1) * cw < N ? (h + 1) * cw : N;
      const int r = 32 * q + lane;
      const int rt = c0 + r;
      for (int col0 = h * cw; col0 < cend; col0 += 8) {
        uint32_t v[8];
        tc_ld_x8(tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(col0), v);
        tc_wait_ld();
        if (r < crows) {
          float x[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int col = col0 + i;
            x[i] = -__uint_as_float(v[i]);
            if (top && rt < ntop && col < n) x[i] += xs[rt * n + col];
          }
          float* qrow = yq + r * n + col0;
          if (col0 + 8 <= n && (reinterpret_cast<uintptr_t>(qrow) & 15) == 0) {
            reinterpret_cast<float4*>(qrow)[0] = make_float4(x[0], x[1], x[2], x[3]);
            reinterpret_cast<float4*>(qrow)[1] = make_float4(x[4], x[5], x[6], x[7]);
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i)
              if (col0 + i < n) qrow[i] = x[i];
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
  if (!ok && pend) mbar_wait_bounded(lbar, lph);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, NC);
}

#endif  // __CUDACC__ && TSQR_TC_KERNELS

}  // namespace tsqr
