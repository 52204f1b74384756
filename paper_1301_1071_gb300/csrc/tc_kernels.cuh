// tc_kernels.cuh -- Step 3 (Sec. III-B) for binary32 data with the product
// Y_i W_i on the 5th-generation tensor cores: tcgen05.mma kind::tf32, operands
// in shared memory, the 128 x N accumulator in tensor memory.  3xTF32 split
// precision: Y = Yh + Yl and W = Wh + Wl with Yh, Yl, Wh, Wl rounded to TF32,
// Y W ~ Yh Wh + Yh Wl + Yl Wh (the dropped Yl Wl is below binary32 rounding).
//
// One CTA per row block (as k_form_q): the tiles of the block are taken last
// to first with X = C (see k_form_q); W of each tile is formed on the CUDA
// cores in binary32, split into the B operands, and the tile's rows are
// processed in chunks of 128 rows: A operands from global memory (split on
// the fly), one MMA chain per chunk (K/8 steps x 3 products), completion on an
// mbarrier, accumulators read back with tcgen05.ld, Q = [X; 0] - D (tile 0)
// or -D written over Y through a shared-memory stage.
//
// Operand layout: no swizzle, K-major: core matrices of 8 rows x 16 bytes
// (4 TF32 values); element (r, k) at ((r/8) * K/4 + k/4) * 128 + (r%8) * 16 +
// (k%4) * 4 bytes, so the descriptor's leading-dimension offset (next core
// along K) is 128 bytes and its stride offset (next 8-row group) K/4 * 128.
#pragma once

#include <cstdint>

#include "device.cuh"
#include "layout.cuh"

namespace tsqr {

constexpr int kTcM = 128;        // rows per MMA chunk (TMEM lanes)
constexpr int kTcThreads = 256;  // 8 warps: warp w reads TMEM lanes 32 (w % 4) ..
constexpr int kTcMaxN = 64;      // largest n on this path
constexpr int kTcMaxE = (kTcMaxN * kTcMaxN + kTcThreads - 1) / kTcThreads;  // W entries per thread

TSQR_HD constexpr int tc_k(int n) { return (n + 7) / 8 * 8; }     // K: MMA K step is 8
TSQR_HD constexpr int tc_n(int n) { return (n + 15) / 16 * 16; }  // N: multiple of 16 at M = 128
TSQR_HD constexpr int tc_cols(int n) { return tc_n(n) <= 32 ? 32 : (tc_n(n) <= 64 ? 64 : 128); }  // TMEM alloc

// Shared-memory layout of k_form_q_tc.  The A buffers double as the stage of
// the n x n operands in the prologue and of the Q rows in the epilogue.
struct FormQTcSmem {
  size_t a_hi, a_lo, b_hi, b_lo, xm, wm, bar, tslot, total;
  TSQR_HD FormQTcSmem(int n) {
    const size_t K = tc_k(n), N = tc_n(n);
    size_t o = 0;
    a_hi = o; o = align_up(o + kTcM * K * 4, 128);
    a_lo = o; o = align_up(o + kTcM * K * 4, 128);
    b_hi = o; o = align_up(o + N * K * 4, 128);
    b_lo = o; o = align_up(o + N * K * 4, 128);
    xm = o; o = align_up(o + (size_t)n * n * 4, 16);
    wm = o; o = align_up(o + (size_t)n * n * 4, 16);
    bar = o; o = align_up(o + 8, 8);
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

// Shared-memory matrix descriptor: start address, leading-dimension and
// stride-dimension byte offsets (all >> 4), fixed field 0b001 at bit 46, no
// swizzle.
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((addr & 0x3FFFF) >> 4) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16) |
         (static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32) | (static_cast<uint64_t>(1) << 46);
}

// Instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1), A and
// B TF32 (bits 7-9 and 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at
// bit 24.
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Step 3, binary32 data, tensor-core product.
//   Yg : m x n (binary32), Y as written by k_local_qr; Q is written over it.
//   Tg : kt slots of n x n binary64 per block (upper triangle).
//   Cg : cblocks blocks of n x n binary64 (cblocks == 1: one C for all).
// Launch: gridDim = p, blockDim = kTcThreads, dynamic smem = FormQTcSmem(n).
__global__ void __launch_bounds__(kTcThreads, 2)
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
  float* stage = a_hi;  // n x n operands (prologue) and Q rows (epilogue); spans a_hi and a_lo
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
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
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  uint32_t parity = 0;
  bool ok = true;
  for (int t = ntiles - 1; t >= 0 && ok; --t) {
    const int tr0 = t == 0 ? 0 : B + (t - 1) * bt;
    const int cnt = t == 0 ? (rows < B ? rows : B) : (rows - tr0 < bt ? rows - tr0 : bt);
    const double* Tb = Tg + (static_cast<int64_t>(blockIdx.x) * kt + t) * nn;
    const float* src = xm;
    float w[kTcMaxE];
    if (t == 0) {
      // Z = Y_top^T X (Y_top unit lower triangular, rows < ntop of the block)
      for (int idx = tid; idx < ntop * n; idx += kTcThreads) stage[idx] = Yg[row0 * n + idx];
      __syncthreads();
#pragma unroll
      for (int e = 0; e < kTcMaxE; ++e) {
        const int idx = tid + e * kTcThreads, kk = idx / n, c = idx % n;
        float acc = 0.0f;
        if (idx < nn && kk < ntop) {
          acc = xm[idx];
          for (int r = kk + 1; r < ntop; ++r) acc = fmaf(stage[r * n + kk], xm[r * n + c], acc);
        }
        w[e] = acc;
      }
      __syncthreads();
#pragma unroll
      for (int e = 0; e < kTcMaxE; ++e)
        if (tid + e * kTcThreads < nn) wm[tid + e * kTcThreads] = w[e];
      __syncthreads();
      src = wm;
    }
    // W = T src (T upper triangular, binary64 slot rounded to binary32)
    for (int idx = tid; idx < nn; idx += kTcThreads) {
      const int i = idx / n, col = idx % n;
      stage[idx] = col >= i ? static_cast<float>(Tb[idx]) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kTcMaxE; ++e) {
      const int idx = tid + e * kTcThreads, kk = idx / n, c = idx % n;
      float acc = 0.0f;
      if (idx < nn)
        for (int i = kk; i < n; ++i) acc = fmaf(stage[kk * n + i], src[i * n + c], acc);
      w[e] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kTcMaxE; ++e) {
      const int idx = tid + e * kTcThreads;
      if (idx < nn) {
        wm[idx] = w[e];
        if (t > 0) xm[idx] -= w[e];  // coefficient of tile t-1
      }
    }
    __syncthreads();
    // B operands: element (c, k) of B^T = W[k][c], split into TF32 hi + lo;
    // warp iteration `it` fills core matrix it (8 rows x 4 values) lane by lane
    for (int it = warp; it < (N / 8) * KQ; it += kTcThreads / 32) {
      const int c = (it / KQ) * 8 + (lane >> 2), k = (it % KQ) * 4 + (lane & 3);
      const float x = (c < n && k < n) ? wm[k * n + c] : 0.0f;
      const float h = tf32_round(x);
      b_hi[it * 32 + lane] = h;
      b_lo[it * 32 + lane] = tf32_round(x - h);
    }

    // the tile's rows, 128 at a time
    const bool top = (t == 0);
    for (int c0 = 0; c0 < cnt && ok; c0 += kTcM) {
      const int crows = cnt - c0 < kTcM ? cnt - c0 : kTcM;
      float* yq = Yg + (row0 + tr0 + c0) * n;  // first row of the chunk (Y in, Q out)
      // A operands from global memory, split into TF32: warp iteration `it`
      // fills core matrix it (rows 8 (it / KQ) .., values 4 (it % KQ) ..) with
      // one float per lane (conflict-free stores; 16-byte row pieces read)
      for (int it = warp; it < (kTcM / 8) * KQ; it += kTcThreads / 32) {
        const int r = (it / KQ) * 8 + (lane >> 2), k = (it % KQ) * 4 + (lane & 3);
        float y = 0.0f;
        if (r < crows && k < n) {
          y = yq[r * n + k];
          if (top && c0 + r < n && k >= c0 + r) y = (k == c0 + r) ? 1.0f : 0.0f;  // unit lower Y_top
        }
        const float h = tf32_round(y);
        a_hi[it * 32 + lane] = h;
        a_lo[it * 32 + lane] = tf32_round(y - h);
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
      // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (rows of the chunk),
      // columns [h N / 2, (h + 1) N / 2) with h = w / 4; Q rows to the stage
      {
        const int q = warp & 3, h = warp >> 2;
        const int r = 32 * q + lane;
        const int rt = c0 + r;  // row within the tile
        for (int col0 = h * (N / 2); col0 < (h + 1) * (N / 2); col0 += 8) {
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
              stage[r * (n + 1) + col] = x;  // odd row stride: no bank conflicts
            }
          }
        }
      }
      tc_fence_before();
      __syncthreads();
      for (int idx = tid; idx < crows * n; idx += kTcThreads) yq[idx] = stage[(idx / n) * (n + 1) + idx % n];
      __syncthreads();  // the stage (A buffers) is free for the next chunk
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NC) : "memory");
}

#endif  // __CUDACC__ && TSQR_TC_KERNELS

}  // namespace tsqr
