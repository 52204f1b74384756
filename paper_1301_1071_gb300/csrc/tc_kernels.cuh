// tc_kernels.cuh -- Step 3 (Sec. III-B) for binary32 data with the product
// Y_i W_i on the 5th-generation tensor cores: tcgen05.mma kind::tf32, operands
// in shared memory, the 128 x N accumulator in tensor memory.  3xTF32 split
// precision: Y = Yh + Yl and W = Wh + Wl with Yh, Yl, Wh, Wl rounded to TF32,
// Y W ~ Yh Wh + Yh Wl + Yl Wh (the dropped Yl Wl is below binary32 rounding).
//
// One CTA per row block (as k_form_q): the tiles of the block are taken last
// to first with X = C (see k_form_q); W of each tile is formed on the CUDA
// cores in binary32, split into the B operands, and the tile's rows are
// processed in chunks of 128 rows: each chunk arrives by bulk copy (TMA) into
// one of two Y buffers while the previous chunk is processed, is split into
// the A operands, multiplied by one MMA chain (K/8 steps x 3 products) that
// completes on an mbarrier, read back from tensor memory with tcgen05.ld, and
// Q = [X; 0] - D (tile 0) or -D is written over Y through the same buffer.
//
// Operand layout: no swizzle, K-major: core matrices of 8 rows x 16 bytes
// (4 TF32 values); element (r, k) at ((r/8) * K/4 + k/4) * 128 + (r%8) * 16 +
// (k%4) * 4 bytes, so the descriptor's leading-dimension offset (next core
// along K) is 128 bytes and its stride offset (next 8-row group) K/4 * 128.
#pragma once

#include <cstdint>

#include "device.cuh"
#include "layout.cuh"
#include "tcgen05.cuh"

namespace tsqr {

constexpr int kTcM = 128;        // rows per MMA chunk (TMEM lanes)
constexpr int kTcThreads = 512;  // 16 warps: warp w reads TMEM lanes 32 (w % 4) ..
constexpr int kTcMaxN = 64;      // largest n on this path
constexpr int kTcMaxE = (kTcMaxN * kTcMaxN + kTcThreads - 1) / kTcThreads;  // W entries per thread

TSQR_HD constexpr int tc_k(int n) { return (n + 7) / 8 * 8; }     // K: MMA K step is 8
TSQR_HD constexpr int tc_n(int n) { return (n + 15) / 16 * 16; }  // N: multiple of 16 at M = 128
TSQR_HD constexpr int tc_cols(int n) { return tc_n(n) <= 32 ? 32 : (tc_n(n) <= 64 ? 64 : 128); }  // TMEM alloc

// Shared-memory layout of k_form_q_tc.  The A buffers double as the stage of
// the n x n operands in the prologue and of the Q rows in the epilogue.
// Y chunks are double-buffered: the bulk copy of the next chunk runs while
// the current one is converted, multiplied and written back.  A Y buffer
// holds 128 rows at row stride n (bulk copy) and later the Q rows at the odd
// stride n + 1 (conflict-free epilogue).
struct FormQTcSmem {
  size_t a_hi, a_lo, b_hi, b_lo, xm, wm, ybuf0, ybuf1, bar, lbar, tslot, total;
  TSQR_HD FormQTcSmem(int n) {
    const size_t K = tc_k(n), N = tc_n(n);
    size_t o = 0;
    a_hi = o; o = align_up(o + kTcM * K * 4, 128);
    a_lo = o; o = align_up(o + kTcM * K * 4, 128);
    b_hi = o; o = align_up(o + N * K * 4, 128);
    b_lo = o; o = align_up(o + N * K * 4, 128);
    xm = o; o = align_up(o + (size_t)n * n * 4, 16);
    wm = o; o = align_up(o + (size_t)n * n * 4, 16);
    ybuf0 = o; o = align_up(o + (size_t)kTcM * (n + 1) * 4, 128);
    ybuf1 = o; o = align_up(o + (size_t)kTcM * (n + 1) * 4, 128);
    bar = o; o = align_up(o + 8, 8);
    lbar = o; o = align_up(o + 16, 8);
    tslot = o; o = align_up(o + 8, 16);
    total = o;
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

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Step 3, binary32 data, tensor-core product.
//   Yg : m x n (binary32), Y as written by k_local_qr; Q is written over it.
//   Tg : kt slots of n x n binary64 per block (upper triangle).
//   Cg : cblocks blocks of n x n binary64 (cblocks == 1: one C for all).
// Launch: gridDim = p, blockDim = kTcThreads, dynamic smem = FormQTcSmem(n).
__global__ void __launch_bounds__(kTcThreads, 1)
    k_form_q_tc(float* Yg, int64_t m, int n, int b, int B, int bt, int kt, const double* __restrict__ Tg,
                const double* __restrict__ Cg, int64_t cblocks, int32_t* status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const FormQTcSmem L(n);
  float* a_hi = reinterpret_cast<float*>(smem + L.a_hi);
  float* a_lo = reinterpret_cast<float*>(smem + L.a_lo);
  float* b_hi = reinterpret_cast<float*>(smem + L.b_hi);
  float* b_lo = reinterpret_cast<float*>(smem + L.b_lo);
  float* xm = reinterpret_cast<float*>(smem + L.xm);
  float* wm = reinterpret_cast<float*>(smem + L.wm);
  float* stage = a_hi;  // n x n operands of the prologue; spans a_hi and a_lo
  float* ybuf[2] = {reinterpret_cast<float*>(smem + L.ybuf0), reinterpret_cast<float*>(smem + L.ybuf1)};
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);    // MMA completion
  uint64_t* lbar = reinterpret_cast<uint64_t*>(smem + L.lbar);  // Y chunk arrival, one per buffer
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.tslot);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int K = tc_k(n), N = tc_n(n), NC = tc_cols(n);
  const int nn = n * n;
  const int64_t row0 = static_cast<int64_t>(blockIdx.x) * b;
  const int rows = static_cast<int>(m - row0 < b ? m - row0 : b);
  const int ntiles = rows <= B ? 1 : 1 + (rows - B + bt - 1) / bt;
  const int ntop = rows < n ? rows : n;
  const uint32_t idesc = tc_idesc_tf32(kTcM, N);
  const int KQ = K / 4;  // core matrices along K
  const uint32_t lbo = 128, sbo = static_cast<uint32_t>(KQ) * 128;

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(lbar, 1);
    mbar_init(lbar + 1, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(NC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  const int64_t cb = cblocks == 1 ? 0 : static_cast<int64_t>(blockIdx.x);
  for (int idx = tid; idx < nn; idx += kTcThreads) xm[idx] = static_cast<float>(Cg[cb * nn + idx]);  // X = C
  // this thread's entries of an n x n product: idx = tid + e kTcThreads = kk n + c
  int ekk[kTcMaxE], ec[kTcMaxE];
  {
    int kk = tid / n, c = tid % n;
    const int dk = kTcThreads / n, dc = kTcThreads % n;
#pragma unroll
    for (int e = 0; e < kTcMaxE; ++e) {
      ekk[e] = kk;
      ec[e] = c;
      kk += dk;
      c += dc;
      if (c >= n) {
        c -= n;
        ++kk;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  // chunk (t, c0): rows [c0, c0 + 128) of tile t; tiles are taken last to
  // first, so the sequence starts at tile ntiles - 1
  auto tile_rows = [&](int t, int& tr0, int& cnt) {
    tr0 = t == 0 ? 0 : B + (t - 1) * bt;
    cnt = t == 0 ? (rows < B ? rows : B) : (rows - tr0 < bt ? rows - tr0 : bt);
  };
  // Issue (thread 0) the bulk copy of the 16-byte-aligned body of chunk
  // (t, c0) into Y buffer s; the rest is read with plain loads on arrival.
  auto issue = [&](int t, int c0, int s) {
    int tr0, cnt;
    tile_rows(t, tr0, cnt);
    const int crows = cnt - c0 < kTcM ? cnt - c0 : kTcM;
    const float* src = Yg + (row0 + tr0 + c0) * n;
    const uint32_t bytes = static_cast<uint32_t>(crows) * n * 4;
    const uint32_t body = (reinterpret_cast<uintptr_t>(src) & 15) == 0 ? (bytes & ~15u) : 0u;
    if (tid == 0 && body > 0) {
      mbar_arrive_expect_tx(lbar + s, body);
      for (uint32_t off = 0; off < body; off += kBulkChunk) {
        const uint32_t len = body - off < kBulkChunk ? body - off : kBulkChunk;
        bulk_g2s(reinterpret_cast<char*>(ybuf[s]) + off, reinterpret_cast<const char*>(src) + off, len, lbar + s);
      }
    }
    return body;
  };

  uint32_t parity = 0, lph[2] = {0u, 0u};
  bool pend[2] = {false, false};  // a bulk copy into the buffer has not been waited for
  bool ok = true;
  int t = ntiles - 1, c0 = 0, cur_tile = -1;
  uint32_t body_cur = issue(t, c0, 0), body_next = 0;
  pend[0] = body_cur > 0;
  for (int ci = 0;; ++ci) {
    const int s = ci & 1;
    int tr0, cnt;
    tile_rows(t, tr0, cnt);
    const int crows = cnt - c0 < kTcM ? cnt - c0 : kTcM;
    float* yq = Yg + (row0 + tr0 + c0) * n;  // first row of the chunk (Y in, Q out)
    const bool top = (t == 0);
    if (t != cur_tile) {
      // ---- prologue of tile t: W, and the B operands
      cur_tile = t;
      const double* Tb = Tg + (static_cast<int64_t>(blockIdx.x) * kt + t) * nn;
      const float* src = xm;
      float w[kTcMaxE];
      if (t == 0) {
        // Z = Y_top^T X (Y_top unit lower triangular, rows < ntop of the block)
        for (int idx = tid; idx < ntop * n; idx += kTcThreads) stage[idx] = Yg[row0 * n + idx];
        __syncthreads();
#pragma unroll
        for (int e = 0; e < kTcMaxE; ++e) {
          const int kk = ekk[e], c = ec[e];
          float acc = 0.0f;
          if (kk < ntop) {
            acc = xm[kk * n + c];
            for (int r = kk + 1; r < ntop; ++r) acc = fmaf(stage[r * n + kk], xm[r * n + c], acc);
          }
          w[e] = acc;
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < kTcMaxE; ++e)
          if (ekk[e] < n) wm[ekk[e] * n + ec[e]] = w[e];
        __syncthreads();
        src = wm;
      }
      // W = T src (T upper triangular, binary64 slot rounded to binary32)
      for (int i = warp; i < n; i += kTcThreads / 32)
        for (int col = lane; col < n; col += 32)
          stage[i * n + col] = col >= i ? static_cast<float>(Tb[i * n + col]) : 0.0f;
      __syncthreads();
#pragma unroll
      for (int e = 0; e < kTcMaxE; ++e) {
        const int kk = ekk[e], c = ec[e];
        float acc = 0.0f;
        if (kk < n)
          for (int i = kk; i < n; ++i) acc = fmaf(stage[kk * n + i], src[i * n + c], acc);
        w[e] = acc;
      }
      __syncthreads();
#pragma unroll
      for (int e = 0; e < kTcMaxE; ++e) {
        if (ekk[e] < n) {
          const int idx = ekk[e] * n + ec[e];
          wm[idx] = w[e];
          if (t > 0) xm[idx] -= w[e];  // coefficient of tile t-1
        }
      }
      __syncthreads();
      // B operands: element (c, k) of B^T = W[k][c], split into TF32 hi + lo;
      // warp iteration `it` fills core matrix it (8 rows x 4 values) lane by lane
      for (int gc = warp; gc < N / 8; gc += kTcThreads / 32)
        for (int kq = 0; kq < KQ; ++kq) {
          const int it = gc * KQ + kq;
          const int c = gc * 8 + (lane >> 2), k = kq * 4 + (lane & 3);
          const float x = (c < n && k < n) ? wm[k * n + c] : 0.0f;
          const float h = tf32_round(x);
          b_hi[it * 32 + lane] = h;
          b_lo[it * 32 + lane] = tf32_round(x - h);
        }

    }
    // ---- prefetch the next chunk into the other buffer (its last readers
    //      finished before the barrier that ended the previous chunk)
    int nt = t, nc0 = c0 + kTcM;
    if (nc0 >= cnt) {
      nt = t - 1;
      nc0 = 0;
    }
    body_next = nt >= 0 ? issue(nt, nc0, s ^ 1) : 0u;
    pend[s ^ 1] = body_next > 0;
    // ---- this chunk's Y: bulk body, then the plain-load remainder
    if (body_cur > 0) {
      ok = mbar_wait_bounded(lbar + s, lph[s]);
      if (ok) {
        lph[s] ^= 1u;
        pend[s] = false;
      }
    }
    for (int e = static_cast<int>(body_cur / 4) + tid; e < crows * n; e += kTcThreads) ybuf[s][e] = yq[e];
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok) {
      if (tid == 0) set_status(status, TSQR_ERR_TIMEOUT);
      break;
    }
    // ---- A operands from the staged rows, split into TF32: warp iteration
    //      `it` fills core matrix it (rows 8 (it / KQ) .., values 4 (it % KQ) ..)
    //      with one value per lane
    {
      const float* ys = ybuf[s];
      for (int gr = warp; gr < kTcM / 8; gr += kTcThreads / 32) {
        const int r = gr * 8 + (lane >> 2);
        const float* yr = ys + r * n + (lane & 3);
        for (int kq = 0; kq < KQ; ++kq) {
          const int it = gr * KQ + kq, k = kq * 4 + (lane & 3);
          float y = 0.0f;
          if (r < crows && k < n) {
            y = yr[kq * 4];
            if (top && c0 + r < n && k >= c0 + r) y = (k == c0 + r) ? 1.0f : 0.0f;  // unit lower Y_top
          }
          const float h = tf32_round(y);
          a_hi[it * 32 + lane] = h;
          a_lo[it * 32 + lane] = tf32_round(y - h);
        }
      }
    }
    fence_proxy_async_smem();  // generic writes of A (and B) -> tensor-core reads
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
      for (int kb = 0; kb < K / 8; ++kb) {
        const uint32_t ko = static_cast<uint32_t>(kb) * 256;
        const uint64_t dah = tc_smem_desc(ah + ko, lbo, sbo), dal = tc_smem_desc(al + ko, lbo, sbo);
        const uint64_t dbh = tc_smem_desc(bh + ko, lbo, sbo), dbl = tc_smem_desc(bl + ko, lbo, sbo);
        tc_mma_tf32(tmem, dah, dbh, idesc, kb > 0);
        tc_mma_tf32(tmem, dah, dbl, idesc, 1);
        tc_mma_tf32(tmem, dal, dbh, idesc, 1);
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
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. (rows of the chunk)
    //      and the h = w / 4 th group of cw columns (cw a multiple of 8: some
    //      groups are empty for small N); Q rows into the chunk's Y buffer at
    //      stride n + 1
    {
      float* qs = ybuf[s];
      const int q = warp & 3, h = warp >> 2;
      const int cw = ((N / 4 + 7) / 8) * 8;
      const int cend = (h + 1) * cw < N ? (h + 1) * cw : N;
      const int r = 32 * q + lane;
      const int rt = c0 + r;  // row within the tile
      for (int col0 = h * cw; col0 < cend; col0 += 8) {
        uint32_t v[8];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
            : "r"(tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(col0)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int col = col0 + i;
          if (col < n && r < crows) {
            float x = -__uint_as_float(v[i]);
            if (top && rt < ntop) x += xm[rt * n + col];
            qs[r * (n + 1) + col] = x;
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    {
      const float* qs = ybuf[s];
      for (int r = warp; r < crows; r += kTcThreads / 32)
        for (int col = lane; col < n; col += 32) yq[r * n + col] = qs[r * (n + 1) + col];
    }
    fence_proxy_async_smem();  // generic reads of this buffer before its next bulk copy
    __syncthreads();
    if (nt < 0) break;
    t = nt;
    c0 = nc0;
    body_cur = body_next;
  }
  // copies still in flight after an error: wait for them (bounded) before
  // the shared memory is released
  for (int s = 0; s < 2; ++s)
    if (!ok && pend[s]) mbar_wait_bounded(lbar + s, lph[s]);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NC) : "memory");
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
#pragma unroll
        for (int e = 0; e < kTcwMaxE; ++e) {
          const int idx = tid + e * kTcThreads;
          if (idx < nn) {
            const int kk = idx / n, i = idx % n;
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
