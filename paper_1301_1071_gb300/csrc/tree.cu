// tree.cu -- the Step-2 tree (Sec. III-B Step 2, Alg. 2) on the structure of
// its nodes, one CTA per node, binary64: the up pass (Householder QR of f
// stacked triangles) and the down pass (the coefficient blocks of a level's
// children from the level's coefficient block C).
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

// P CTAs per node, CTA (node, panel) for the panel's column groups (the
// columns of W = T C and of the node's Q blocks are independent, so a level
// of few nodes still fills the GPU).  Y: the level's input stack (rows x n,
// binary64), node b = rows [b f n, min((b + 1) f n, rows)); T: one n x n slot
// per node (upper triangle); C: cblocks coefficient blocks (cblocks == 1: all
// nodes use C).  A thread group of ceil(n/2) row pairs x ncp column groups
// (CJ columns each) forms the panel of one n x n product; KB groups take KB
// blocks of the node at once (small n: the 24 further blocks of a 25-way node
// at n = 25 take 3 passes, not 24).  Group 0 forms W.  Threads: KB x group
// size <= MAXT.
template <int CJ, int MAXT>
__global__ void __launch_bounds__(MAXT) k_tree_down(double* Y, int64_t rows, int n, int f, const double* T,
                                                    const double* C, int64_t cblocks, int KB, int P) {
  extern __shared__ __align__(16) double tsm[];
  const int ncg = (n + CJ - 1) / CJ;
  const int ncp = (ncg + P - 1) / P;  // column groups per panel
  const int ld = ncg * CJ + 1;
  const int gsz = (n + 1) / 2 * ncp;  // threads per group
  double* Wb = tsm;                   // T, then W = T C (the panel's columns)
  const int tid = threadIdx.x, NT = blockDim.x;
  const int grp = tid / gsz, gt = tid - grp * gsz;
  double* Bb = tsm + (1 + (grp < KB ? grp : 0)) * n * ld;  // the group's block (group 0's holds C first)
  const int64_t node = blockIdx.x / P;
  const int pnl = static_cast<int>(blockIdx.x - node * P);
  const int cb0 = pnl * ncp * CJ;                           // the panel's first column
  const int cb1 = (pnl + 1) * ncp * CJ < n ? (pnl + 1) * ncp * CJ : n;  // ... and its end (<= cb0: none)
  const int64_t r0 = node * f * n;
  const int nb = static_cast<int>((rows - r0) / n < f ? (rows - r0) / n : f);
  const double* Tn = T + node * n * n;
  const double* Cn = C + (cblocks == 1 ? 0 : node * n * n);
  double* Yn = Y + r0 * n;
  double* B0 = tsm + n * ld;
  // T (upper triangle; the slot's lower part is not defined) and C, copied
  // asynchronously (every thread's copies in flight at once; the zeros
  // around them are plain stores)
  for (int idx = tid; idx < n * ld; idx += NT) {
    const int i = idx / ld, c = idx - i * ld;
    if (c < n && c >= i) cp_async_8(Wb + idx, Tn + i * n + c);
    else Wb[idx] = 0.0;
    if (c < n) cp_async_8(B0 + idx, Cn + i * n + c);
    else B0[idx] = 0.0;
  }
  cp_async_wait_all();
  __syncthreads();
  const int g = gt / ncp, cg = gt - g * ncp;
  const bool active = grp < KB;  // every thread of a group has a row pair
  // the thread's column group; the last panel may have fewer (or none)
  const bool colok = pnl * ncp + cg < ncg;
  const int c0 = cb0 + cg * CJ;
  double top[CJ], bot[CJ];
  // W = T C (group 0, the panel's columns)
  if (grp == 0 && colok) tri_rows<CJ>(Wb, B0, ld, n, g, c0, top, bot);
  __syncthreads();
  if (grp == 0 && colok) {
#pragma unroll
    for (int b = 0; b < CJ; ++b) {
      Wb[g * ld + c0 + b] = top[b];
      if (n - 1 - g != g) Wb[(n - 1 - g) * ld + c0 + b] = bot[b];
    }
  }
  __syncthreads();
  // block 1 of the node: C - W (the panel's columns)
  const int pw = cb1 > cb0 ? cb1 - cb0 : 0;
  for (int idx = tid; idx < n * pw; idx += NT) {
    const int i = idx / pw, c = cb0 + idx - i * pw;
    Yn[i * n + c] = B0[i * ld + c] - Wb[i * ld + c];
  }
  // blocks 2..nb: -V_k W, KB at a time (V_k staged whole before its rows
  // are overwritten; the node's other panels stage their own copies before
  // writing their own columns only)
  for (int kb = 1; kb < nb; kb += KB) {
    const int k = kb + grp;
    const bool mine = active && k < nb;
    double* Yk = Yn + static_cast<int64_t>(k) * n * n;
    __syncthreads();  // the buffers are free (previous pass's reads are done)
    if (mine) {
      for (int idx = gt; idx < n * ld; idx += gsz) {
        const int i = idx / ld, c = idx - i * ld;
        if (c < n && c >= i) cp_async_8(Bb + idx, Yk + i * n + c);
        else Bb[idx] = 0.0;
      }
    }
    cp_async_wait_all();
    __syncthreads();
    // every panel of the node has staged these blocks before any overwrites
    // its columns of them (the node's P CTAs are one cluster)
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
    if (mine && colok) {
      tri_rows<CJ>(Bb, Wb, ld, n, g, c0, top, bot);
#pragma unroll
      for (int b = 0; b < CJ; ++b) {
        if (c0 + b < cb1) {
          Yk[g * n + c0 + b] = -top[b];
          if (n - 1 - g != g) Yk[(n - 1 - g) * n + c0 + b] = -bot[b];
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Up pass: Householder QR of a node [R_1; ...; R_f] (f upper-triangular n x n
// blocks; the last node may have fewer).  Column j's reflector involves row
// j of R_1 and rows 0..j of every other block -- the other entries of the
// column are zero and stay zero (no reflector reaches them) -- so each column
// step costs (f - 1)(j + 1)(n - j) FMAs for the dots and as many for the
// update, where the dense factorisation of the f n x n node costs f n (n - j).
// Reflector convention as the row-block kernel: for the column's squared norm
// S and its pivot alpha, beta = -copysign(sqrt(S), alpha), v = x / (alpha -
// beta) with v_j = 1, tau = (beta - alpha) / beta; a zero column gives the
// identity (tau = 0).  Outputs as the row-block kernel's: the node's R (raw
// signs, zeros below the diagonal) into Rout's block, the Householder vectors
// over the node's rows of Y (blocks 2..f; block 1 holds R and is never read),
// tau_j and the Gram entries v_i^T v_j (i < j) into the node's T slot
// (k_build_t forms T).  WANT_Y = false: R only.
// Threads: G per column (G a power of two, the G lanes of a column in one
// warp), column c = tid / G; the lanes of a group split the column's
// sub-column (all blocks, rows 0..j) as one index space.  Per column j two
// CTA barriers: column j's group forms the norm, the reflector scalars and v
// (its G lanes reduce by shuffles); then every later column's group forms its
// dot with v and its update -- each column is touched by its own group only,
// so the dots and the update of a column need no barrier between them.
// The node sits in shared memory, row r at M[r * ldm].
template <bool WANT_Y>
__global__ void __launch_bounds__(1024) k_tree_up(const double* X, int64_t rows, int n, int f, double* Y,
                                                  double* Rout, double* Tst, int G) {
  extern __shared__ __align__(16) double usm[];
  const int ldm = n + 1;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int c = tid / G, u = tid - c * G;  // my column and my lane within its group
  const int64_t node = blockIdx.x;
  const int64_t r0 = node * f * n;
  const int nb = static_cast<int>((rows - r0) / n < f ? (rows - r0) / n : f);
  double* M = usm;                      // nb n rows
  double* taus = M + nb * n * ldm;      // tau per column
  const double* Xn = X + r0 * n;
  for (int idx = tid; idx < nb * n * n; idx += NT) {
    const int r = idx / n, cc = idx - r * n;
    M[r * ldm + cc] = cc >= r % n ? Xn[idx] : 0.0;  // the blocks are triangular; below: exact zeros
  }
  __syncthreads();
  const int nsub = nb - 1;  // blocks below the first
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((tid & 31) & ~(G - 1)));
  for (int j = 0; j < n; ++j) {
    // the sub-column of column j: entries e = 0 .. nsub (j + 1) - 1, block
    // k = 1 + e / (j + 1), row lr = e % (j + 1); lane u takes e = u, u + G, ..
    // (stepped without division: G = dq (j + 1) + dr)
    const int len = j + 1, ne = nsub * len;
    const int dq = G / len, dr = G - dq * len;
    const int k0 = 1 + u / len, l0 = u - (u / len) * len;
    if (c == j) {
      double ss = 0.0;
      {
        int k = k0, lr = l0;
        for (int e = u; e < ne; e += G) {
          const double v = M[(k * n + lr) * ldm + j];
          ss = fma(v, v, ss);
          lr += dr;
          k += dq;
          if (lr >= len) {
            lr -= len;
            ++k;
          }
        }
      }
      for (int o = G >> 1; o > 0; o >>= 1) ss += __shfl_xor_sync(gmask, ss, o);
      const double alpha = M[j * ldm + j];
      const double sigma = sqrt(fma(alpha, alpha, ss));
      double beta, scal, tau;
      if (sigma == 0.0) {
        beta = alpha;
        scal = 0.0;
        tau = 0.0;
      } else {
        beta = alpha >= 0.0 ? -sigma : sigma;
        scal = 1.0 / (alpha - beta);
        tau = (beta - alpha) / beta;
      }
      {  // v: the scaled sub-column
        int k = k0, lr = l0;
        for (int e = u; e < ne; e += G) {
          M[(k * n + lr) * ldm + j] *= scal;
          lr += dr;
          k += dq;
          if (lr >= len) {
            lr -= len;
            ++k;
          }
        }
      }
      if (u == 0) {
        taus[j] = tau;
        M[j * ldm + j] = beta;
      }
    }
    __syncthreads();
    const double tau = taus[j];
    if (c > j && c < n && tau != 0.0) {
      // w_c = a_jc + v^T a_c over the sub-column rows; a_c -= (tau w_c) v
      double w = 0.0;
      {
        int k = k0, lr = l0;
        for (int e = u; e < ne; e += G) {
          const double* row = M + (k * n + lr) * ldm;
          w = fma(row[j], row[c], w);
          lr += dr;
          k += dq;
          if (lr >= len) {
            lr -= len;
            ++k;
          }
        }
      }
      for (int o = G >> 1; o > 0; o >>= 1) w += __shfl_xor_sync(gmask, w, o);
      const double tw = tau * (M[j * ldm + c] + w);
      if (u == 0) M[j * ldm + c] -= tw;
      {
        int k = k0, lr = l0;
        for (int e = u; e < ne; e += G) {
          double* row = M + (k * n + lr) * ldm;
          row[c] = fma(-tw, row[j], row[c]);
          lr += dr;
          k += dq;
          if (lr >= len) {
            lr -= len;
            ++k;
          }
        }
      }
    }
    __syncthreads();
  }
  // R of the node (raw signs)
  double* Rn = Rout + node * n * n;
  for (int idx = tid; idx < n * n; idx += NT) {
    const int i = idx / n, cc = idx - i * n;
    Rn[idx] = cc >= i ? M[i * ldm + cc] : 0.0;
  }
  if constexpr (WANT_Y) {
    // Householder vectors over the node's rows (block 1: R, never read)
    double* Yn = Y + r0 * n;
    for (int idx = tid; idx < nb * n * n; idx += NT) {
      const int r = idx / n, cc = idx - r * n;
      Yn[idx] = M[r * ldm + cc];
    }
    // tau and the Gram entries G(i, c) = sum_k sum_{lr <= i} v_i(lr) v_c(lr), i < c
    double* Tn = Tst + node * n * n;
    for (int idx = tid; idx < n * n; idx += NT) {
      const int i = idx / n, cc = idx - i * n;
      if (cc < i) continue;
      double g = taus[i];
      if (cc > i) {
        g = 0.0;
        for (int k = 1; k < nb; ++k) {
          const double* blk = M + static_cast<size_t>(k) * n * ldm;
          for (int lr = 0; lr <= i; ++lr) g = fma(blk[lr * ldm + i], blk[lr * ldm + cc], g);
        }
      }
      Tn[idx] = g;
    }
  }
}


// ---------------------------------------------------------------------------
// Up pass over a cluster, for nodes of f <= kTreeClMaxF triangles too large
// for one CTA's shared memory (n > 84 at f = 4): CTA q of the node's cluster
// holds block q (block 0 = R_1).  The factorisation is the one above with
// each column's sums split by block and one cluster barrier per column.
// Column j's vector is v = scal x (x: the column's entries below the pivot,
// scal = 1 / (alpha - beta)), so every sum it enters can be formed from x
// before scal is known:
//   (1) column j's lanes form their block's squared norm of x, every later
//       column c's lanes their block's dot x^T a_c (block 0 instead: the
//       pivot alpha and the pivot row's entries a_jc); lane u of a group
//       stores its group's partial into the receive buffers of CTAs u,
//       u + G, .. (remote stores), so every CTA receives all f partials;
//   (2) cluster barrier;
//   (3) column j's lanes sum the f norm partials they received in a fixed
//       shuffle order (so every CTA forms the same beta, scal and tau) and
//       publish the scalars; CTA barrier; every later group sums its dot
//       partials the same way, w_c = a_jc + scal sum_k x_k^T a_c, and
//       a_c -= tau w_c v over the group's own rows; CTA barrier (column
//       j + 1 has been updated).
// The receive buffers alternate by the parity of j: a CTA refills one only
// after the next barrier, which every CTA reaches after its reads of it.
// x is kept unscaled during the loop (no later column reads it) and scaled
// into v at the end.  The Gram entries of T are summed by block and then
// over the ranks in order, in chunks of gch rows.  Outputs as k_tree_up.
// Threads: G = 4 lanes per column, column c = tid / G: few lanes keep the
// shuffle trees (binary64 adds) short, and with a Gram chunk of 16 rows two
// CTAs fit an SM (levels of many nodes run in half the waves).
template <bool WANT_Y>
__global__ void __launch_bounds__(1024) k_tree_up_cl(const double* X, int64_t rows, int n, int f, double* Y,
                                                     double* Rout, double* Tst, int G, int gch) {
  extern __shared__ __align__(16) double usm[];
  const int ldm = n + 1, ldp = n + 2;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int c = tid / G, u = tid - c * G;
  const int q = static_cast<int>(cluster_ctarank());
  const int64_t node = blockIdx.x / f;
  const int64_t r0 = node * f * n;
  const int nb = static_cast<int>((rows - r0) / n < f ? (rows - r0) / n : f);
  const bool lower = q > 0 && q < nb;  // a block below the first (the last node may have fewer)
  double* M = usm;                     // this CTA's block, row r at M[r * ldm]
  double* part = M + n * ldm;          // [2][f][n + 2]: partials received from rank r (column c; n: norm, n + 1: alpha)
  double* taus = part + 2 * f * ldp;   // tau per column
  double* scals = taus + n;            // 1 / (alpha - beta) per column
  double* gp = scals + n;              // partial Gram rows, gch x n
  if (q < nb) {
    const double* Xb = X + (r0 + static_cast<int64_t>(q) * n) * n;
    for (int idx = tid; idx < n * n; idx += NT) {
      const int r = idx / n, cc = idx - r * n;
      M[r * ldm + cc] = cc >= r ? Xb[idx] : 0.0;
    }
  }
  __syncthreads();
  cluster_barrier();  // every CTA of the cluster has started (its receive buffers exist)
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((tid & 31) & ~(G - 1)));
  for (int j = 0; j < n; ++j) {
    double* pb = part + (j & 1) * f * ldp;
    // (1) partials of column j's norm (group j) and of the dots x^T a_c (groups c > j)
    if (c >= j && c < n) {
      double s = 0.0;
      if (lower)
        for (int lr = u; lr <= j; lr += G) s = fma(M[lr * ldm + j], M[lr * ldm + c], s);
      for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o);
      if (q == 0) s = M[j * ldm + c];  // block 0: alpha (c == j) or a_jc
      for (int r = u; r < f; r += G) st_cluster(cluster_map(pb + q * ldp + (c == j ? n : c), static_cast<uint32_t>(r)), s);
    }
    cluster_barrier();
    // (3) the reflector from the received partials (column j's lanes: one
    //     sqrt and two divisions per CTA; binary64 division is costly on
    //     this part), then the update
    if (c == j) {
      // ranks >= 1 summed in a fixed order: lane u takes ranks u, u + G, ..,
      // then a shuffle tree
      double ss = 0.0;
      for (int r = u > 0 ? u : G; r < f; r += G) ss += pb[r * ldp + n];
      for (int o = G >> 1; o > 0; o >>= 1) ss += __shfl_xor_sync(gmask, ss, o);
      const double alpha = pb[n];  // rank 0's slot for column j
      const double sigma = sqrt(fma(alpha, alpha, ss));
      double beta, scal, tau;
      if (sigma == 0.0) {
        beta = alpha;
        scal = 0.0;
        tau = 0.0;
      } else {
        beta = alpha >= 0.0 ? -sigma : sigma;
        scal = 1.0 / (alpha - beta);
        tau = (beta - alpha) / beta;
      }
      if (u == 0) {
        taus[j] = tau;
        scals[j] = scal;
        if (q == 0) M[j * ldm + j] = beta;
      }
    }
    __syncthreads();
    const double tau = taus[j];
    if (c > j && c < n && tau != 0.0) {
      const double scal = scals[j];
      double sd = 0.0;
      for (int r = u > 0 ? u : G; r < f; r += G) sd += pb[r * ldp + c];
      for (int o = G >> 1; o > 0; o >>= 1) sd += __shfl_xor_sync(gmask, sd, o);
      const double tw = tau * fma(scal, sd, pb[c]);  // pb[c]: rank 0's a_jc
      if (q == 0) {
        if (u == 0) M[j * ldm + c] -= tw;
      } else if (lower) {
        const double ts = tw * scal;
        for (int lr = u; lr <= j; lr += G) M[lr * ldm + c] = fma(-ts, M[lr * ldm + j], M[lr * ldm + c]);
      }
    }
    __syncthreads();  // column j + 1's entries are read by every later group
  }
  // v = scal x over the lower blocks
  if (lower)
    for (int idx = tid; idx < n * n; idx += NT) {
      const int r = idx / n, cc = idx - r * n;
      if (r <= cc) M[r * ldm + cc] *= scals[cc];
    }
  __syncthreads();
  if (q == 0) {
    double* Rn = Rout + node * n * n;
    for (int idx = tid; idx < n * n; idx += NT) {
      const int i = idx / n, cc = idx - i * n;
      Rn[idx] = cc >= i ? M[i * ldm + cc] : 0.0;
    }
  }
  if constexpr (WANT_Y) {
    if (q < nb) {
      double* Yb = Y + (r0 + static_cast<int64_t>(q) * n) * n;
      for (int idx = tid; idx < n * n; idx += NT) {
        const int r = idx / n, cc = idx - r * n;
        Yb[idx] = M[r * ldm + cc];
      }
    }
    // tau and the Gram entries G(i, c) = sum_k sum_{lr <= i} v_i(lr) v_c(lr), i < c
    double* Tn = Tst + node * n * n;
    for (int i0 = 0; i0 < n; i0 += gch) {
      const int nr = n - i0 < gch ? n - i0 : gch;
      for (int e = tid; e < nr * n; e += NT) {
        const int i = i0 + e / n, cc = e - (e / n) * n;
        double g = 0.0;
        if (lower && cc > i)
          for (int lr = 0; lr <= i; ++lr) g = fma(M[lr * ldm + i], M[lr * ldm + cc], g);
        gp[e] = g;
      }
      cluster_barrier();
      for (int e = q * NT + tid; e < nr * n; e += f * NT) {
        const int i = i0 + e / n, cc = e - (e / n) * n;
        if (cc < i) continue;
        double g = taus[i];
        if (cc > i) {
          double pr[kTreeClMaxF];
#pragma unroll
          for (int r = 0; r < kTreeClMaxF; ++r) pr[r] = r < f ? ld_cluster(cluster_map(gp + e, r)) : 0.0;
          g = 0.0;
#pragma unroll
          for (int r = 0; r < kTreeClMaxF; ++r) g += pr[r];
        }
        Tn[i * n + cc] = g;
      }
      cluster_barrier();  // gp is refilled by the next chunk (and read until here)
    }
  } else {
    cluster_barrier();  // no CTA leaves while another may still store into its buffers
  }
}

}  // namespace

cudaError_t launch_tree_down(double* Y, int64_t rows, int n, int f, int64_t p, const double* T, const double* C,
                             int64_t cblocks, cudaStream_t st) {
  const int CJ = n > 50 ? 10 : 5;
  const int maxt = CJ == 10 ? 512 : 1024;
  const int ncg = (n + CJ - 1) / CJ;
  const int ld = ncg * CJ + 1;
  // panels per node: a level of few nodes is spread over clusters of up to
  // 5 CTAs (column panels); a wide level keeps one CTA per node
  int P = 1;
  while (P < 5 && P < ncg && p * P < 2 * kDefaultSMs) ++P;
  const int ncp = (ncg + P - 1) / P;
  const int gsz = (n + 1) / 2 * ncp;
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
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(p * P));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(P);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, Y, rows, n, f, T, C, cblocks, KB, P);
}

size_t tree_up_smem(int n, int f) {
  return (static_cast<size_t>(f) * n * (n + 1) + n) * sizeof(double);
}

bool tree_up_fits(int n, int f) { return f >= 2 && tree_up_smem(n, f) <= kSmemMax; }

cudaError_t launch_tree_up(const double* X, int64_t rows, int n, int f, int64_t p, double* Y, double* Rout,
                           double* Tst, cudaStream_t st) {
  if (!tree_up_fits(n, f)) return cudaErrorInvalidConfiguration;
  const size_t smem = tree_up_smem(n, f);
  // lanes per column: a power of two from 4 to 32, about two sub-column
  // blocks per lane (a column's work grows with the node's f - 1 lower
  // blocks), at most 1024 threads
  int G = 4;
  while (G < 32 && G < 2 * (f - 1) && 2 * G * n <= 1024) G *= 2;
  const int NT = (G * n + 31) / 32 * 32;
  auto fn = Y ? k_tree_up<true> : k_tree_up<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)p, NT, smem, st>>>(X, rows, n, f, Y, Rout, Tst, G);
  return cudaGetLastError();
}

static size_t tree_up_cl_smem(int n, int gch) {
  return (static_cast<size_t>(n) * (n + 1) + 2 * static_cast<size_t>(kTreeClMaxF) * (n + 2) +
          2 * static_cast<size_t>(n) + static_cast<size_t>(gch) * n) *
         sizeof(double);
}

// Gram rows per chunk of the cluster up pass: 16, fewer where two CTAs per
// SM would not fit otherwise, at least 8
static int tree_up_cl_gch(int n) {
  int g = 16;
  while (g > 8 && 2 * (tree_up_cl_smem(n, g) + 1024) > kSmemPerSM) g -= 8;
  return g;
}

// lanes per column (4; 0: the node's columns exceed 1024 threads)
static int tree_up_cl_lanes(int n, int) { return 4 * n <= 1024 ? 4 : 0; }

bool tree_up_cl_fits(int n, int f) {
  return f >= 2 && f <= kTreeClMaxF && tree_up_cl_lanes(n, f) > 0 &&
         tree_up_cl_smem(n, tree_up_cl_gch(n)) <= kSmemMax;
}

cudaError_t launch_tree_up_cl(const double* X, int64_t rows, int n, int f, int64_t p, double* Y, double* Rout,
                              double* Tst, cudaStream_t st) {
  if (!tree_up_cl_fits(n, f)) return cudaErrorInvalidConfiguration;
  const int gch = tree_up_cl_gch(n);
  const size_t smem = tree_up_cl_smem(n, gch);
  const int G = tree_up_cl_lanes(n, f);
  const int NT = (G * n + 31) / 32 * 32;
  auto fn = Y ? k_tree_up_cl<true> : k_tree_up_cl<false>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(p * f));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(f);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, X, rows, n, f, Y, Rout, Tst, G, gch);
}

}  // namespace tsqr
