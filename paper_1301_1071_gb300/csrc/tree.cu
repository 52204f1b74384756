// tree.cu -- the Step-2 tree's down pass (Sec. III-B Step 2, Alg. 2): the
// coefficient blocks of a level's children from the level's coefficient
// block C, one CTA per tree node, binary64.
//
// A tree node stacks f upper-triangular R factors, [R_1; ...; R_f].  Its
// Householder vectors keep that structure exactly: the entries of R_1 below
// the diagonal are zero and no reflector touches them, so the first block of
// Y is the identity, and reflector j touches rows 0..j of every other block,
// so Y = [I; V_2; ...; V_f] with each V_k upper triangular.  The node's Q
// applied to [C; 0] is then
//   W = T C,  Q = [C - W; -V_2 W; ...; -V_f W]
// (T upper triangular): n^3/2 FMAs for W and n^3/2 per further block, where
// the general Step-3 product (Y_top^T C, T, and the dense Y W) takes
// n^3 (3/2 + f).  Q is written over the node's rows of Y.
#include <cstdint>
#include <cuda_runtime.h>

#include "device.cuh"
#include "launch.h"

namespace tsqr {

namespace {

// acc(r, c0 + b) = sum_{j >= r} U(r, j) D(j, c0 + b) for the thread's two
// rows r = g (top) and n-1-g (bottom): n + 1 steps per thread whatever g is,
// so every thread of the CTA runs the same count.  U and D in shared memory
// (leading dimension ld); D's columns n..CJ*ceil(n/CJ)-1 are zero.
template <int CJ>
__device__ __forceinline__ void tri_rows(const double* U, const double* D, int ld, int n, int g, int c0,
                                         double (&top)[CJ], double (&bot)[CJ]) {
#pragma unroll
  for (int b = 0; b < CJ; ++b) top[b] = bot[b] = 0.0;
  const int rt = g, rb = n - 1 - g;
  for (int j = rt; j < n; ++j) {
    const double u = U[rt * ld + j];
    const double* dr = D + j * ld + c0;
#pragma unroll
    for (int b = 0; b < CJ; ++b) top[b] = fma(u, dr[b], top[b]);
  }
  if (rb != rt) {
    for (int j = rb; j < n; ++j) {
      const double u = U[rb * ld + j];
      const double* dr = D + j * ld + c0;
#pragma unroll
      for (int b = 0; b < CJ; ++b) bot[b] = fma(u, dr[b], bot[b]);
    }
  }
}

// One CTA per node.  Y: the level's input stack (rows x n, binary64), node b
// = rows [b f n, min((b + 1) f n, rows)); T: one n x n slot per node (upper
// triangle); C: cblocks coefficient blocks (cblocks == 1: all nodes use C).
// A thread group of ceil(n/2) row pairs x ceil(n/CJ) column groups forms one
// n x n product; KB groups take KB blocks of the node at once (small n:
// the 24 further blocks of a 25-way node at n = 25 take 3 passes, not 24).
// Group 0 forms W.  Threads: KB x group size <= MAXT.
template <int CJ, int MAXT>
__global__ void __launch_bounds__(MAXT) k_tree_down(double* Y, int64_t rows, int n, int f, const double* T,
                                                    const double* C, int64_t cblocks, int KB) {
  extern __shared__ __align__(16) double tsm[];
  const int ncg = (n + CJ - 1) / CJ;
  const int ld = ncg * CJ + 1;
  const int gsz = (n + 1) / 2 * ncg;  // threads per group
  double* Wb = tsm;                   // T, then W = T C
  const int tid = threadIdx.x, NT = blockDim.x;
  const int grp = tid / gsz, gt = tid - grp * gsz;
  double* Bb = tsm + (1 + (grp < KB ? grp : 0)) * n * ld;  // the group's block (group 0's holds C first)
  const int64_t node = blockIdx.x;
  const int64_t r0 = node * f * n;
  const int nb = static_cast<int>((rows - r0) / n < f ? (rows - r0) / n : f);
  const double* Tn = T + node * n * n;
  const double* Cn = C + (cblocks == 1 ? 0 : node * n * n);
  double* Yn = Y + r0 * n;
  double* B0 = tsm + n * ld;
  // T (upper triangle; the slot's lower part is not defined) and C
  for (int idx = tid; idx < n * ld; idx += NT) {
    const int i = idx / ld, c = idx - i * ld;
    Wb[idx] = (c < n && c >= i) ? Tn[i * n + c] : 0.0;
    B0[idx] = c < n ? Cn[i * n + c] : 0.0;
  }
  __syncthreads();
  const int g = gt / ncg, cg = gt - g * ncg;
  const bool active = grp < KB;  // every thread of a group has a row pair
  const int c0 = cg * CJ;
  double top[CJ], bot[CJ];
  // W = T C (group 0)
  if (grp == 0) tri_rows<CJ>(Wb, B0, ld, n, g, c0, top, bot);
  __syncthreads();
  if (grp == 0) {
#pragma unroll
    for (int b = 0; b < CJ; ++b) {
      Wb[g * ld + c0 + b] = top[b];
      if (n - 1 - g != g) Wb[(n - 1 - g) * ld + c0 + b] = bot[b];
    }
  }
  __syncthreads();
  // block 1 of the node: C - W
  for (int idx = tid; idx < n * n; idx += NT) {
    const int i = idx / n, c = idx - i * n;
    Yn[idx] = B0[i * ld + c] - Wb[i * ld + c];
  }
  // blocks 2..nb: -V_k W, KB at a time (V_k staged whole before its rows
  // are overwritten)
  for (int kb = 1; kb < nb; kb += KB) {
    const int k = kb + grp;
    const bool mine = active && k < nb;
    double* Yk = Yn + static_cast<int64_t>(k) * n * n;
    __syncthreads();  // the buffers are free (previous pass's reads are done)
    if (mine) {
      for (int idx = gt; idx < n * ld; idx += gsz) {
        const int i = idx / ld, c = idx - i * ld;
        Bb[idx] = (c < n && c >= i) ? Yk[i * n + c] : 0.0;
      }
    }
    __syncthreads();
    if (mine) {
      tri_rows<CJ>(Bb, Wb, ld, n, g, c0, top, bot);
#pragma unroll
      for (int b = 0; b < CJ; ++b) {
        if (c0 + b < n) {
          Yk[g * n + c0 + b] = -top[b];
          if (n - 1 - g != g) Yk[(n - 1 - g) * n + c0 + b] = -bot[b];
        }
      }
    }
  }
}

}  // namespace

cudaError_t launch_tree_down(double* Y, int64_t rows, int n, int f, int64_t p, const double* T, const double* C,
                             int64_t cblocks, cudaStream_t st) {
  const int CJ = n > 50 ? 10 : 5;
  const int maxt = CJ == 10 ? 512 : 1024;
  const int ncg = (n + CJ - 1) / CJ;
  const int ld = ncg * CJ + 1;
  const int gsz = (n + 1) / 2 * ncg;
  const size_t buf = static_cast<size_t>(n) * ld * sizeof(double);
  if (gsz > maxt || 2 * buf > kSmemMax) return cudaErrorInvalidConfiguration;
  // groups: as many further blocks at once as threads and shared memory allow
  int KB = maxt / gsz;
  if (KB > f - 1) KB = f - 1;
  if (KB < 1) KB = 1;
  while (KB > 1 && (1 + KB) * buf > kSmemMax) --KB;
  const int NT = (KB * gsz + 31) / 32 * 32;
  const size_t smem = (1 + KB) * buf;
  auto fn = CJ == 10 ? k_tree_down<10, 512> : k_tree_down<5, 1024>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)p, NT, smem, st>>>(Y, rows, n, f, T, C, cblocks, KB);
  return cudaGetLastError();
}

}  // namespace tsqr
