// plan.h -- host-side plan of a direct-TSQR call: kernel configuration per
// dtype and n, row-block partition (Step 1), recursive tree levels (Step 2,
// Alg. 2) and the workspace layout.  Pure host code, unit-testable.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

namespace tsqr {

constexpr int kNpc = 5;                // columns per thread (register tile width)
constexpr size_t kSmemMax = 232448;    // 227 KB dynamic shared memory per CTA
constexpr size_t kSmemPerSM = 233472;  // 228 KB per SM, 1 KB of it reserved per CTA
constexpr size_t kHeaderBytes = 256;   // status word + padding at the start of work

// Kernel kind of a tall pass: storage / compute types.
enum KernelKind { kKindF64 = 0, kKindF32 = 1, kKindDF64 = 2 };

struct KernelCfg {
  int kind = kKindF64;
  int npc = kNpc;
  int R = 0;    // rows per thread
  int CS = 0;   // column slices (warps per row group)
  int NRG = 0;  // row groups of 32 rows
  int NT = 0;   // threads per CTA = 32 * CS * NRG
  int B = 0;    // rows per CTA capacity = 32 * NRG * R
  size_t smem_qr = 0, smem_fq = 0;
  int tile = 0;     // index of the register tile (kern_f64.cu / kern_f32.cu)
  int fq_rows = 0;  // rows per staged chunk of k_form_q (<= B)
  int rm_rows = 0;  // staged rows per CTA of k_rowmul (<= B; halves hold two inputs)
  size_t smem_rm = 0;
  int ctas = 1;     // CTAs of k_local_qr resident per SM (registers, shared memory)
  // k_form_q / k_rowmul walk the columns of their staged rows in a per-lane
  // rotated order (lane l starts at column l mod n): with a row stride of n
  // elements the lanes of a warp (consecutive rows) otherwise hit the same
  // shared-memory bank when n x element size is a multiple of 32 bytes
  int skew = 0;
};

// Default tile policies: kPolicyStep1 takes the largest spill-free register
// tile (ties: fewer threads; used for double-float Step 1 and, with at least
// 2n rows so that a node merges two or more R factors, for the tree);
// kPolicyLargest takes the largest block; kPolicyInFlight takes the most rows
// resident per SM (B x CTAs per SM), ties going to more CTAs: two CTAs of one
// row group each (the look-ahead loop) overlap their per-column barriers and
// reductions, which one CTA of two row groups cannot (binary64 and binary32
// Step 1).
enum { kPolicyStep1 = 0, kPolicyLargest = 1, kPolicyInFlight = 2 };

// Picks the register tile of kernel kind `kind` for n (want_b > 0: the
// smallest per-CTA capacity that holds want_b rows; else `policy`).
bool choose_cfg(int kind, int n, KernelCfg* out, int64_t want_b = 0, int policy = kPolicyStep1, int min_b = 0);

struct Level {
  int64_t rows = 0;  // rows of this level's input matrix
  int64_t b = 0;     // rows per block
  int64_t p = 0;     // number of blocks
  // a block taller than the register tile (b > B) is factored as a flat
  // tree of tiles inside one CTA: B rows, then bt rows per tile, kt tiles at
  // most (kt T slots per block)
  int64_t bt = 0;
  int kt = 1;
  size_t off_S = 0;  // byte offset of the p blocks of R (n x n, binary64)
  size_t off_T = 0;  // byte offset of the p kt T slots (n x n, binary64)
};

struct Plan {
  int64_t m = 0, n = 0;
  int esz = 8;           // element size of the tall matrices
  KernelCfg cfg0;        // Step-1 kernel config (dtype of A)
  KernelCfg cfg64;       // tree kernel config (binary64)
  int prec = 0;          // the resolved tsqr_prec (TSQR_PREC_AUTO taken)
  bool tc3 = false;      // Step 3 on the tensor cores (3xTF32, binary32 data)
  bool oz3 = false;      // Step 3 on the tensor cores (Ozaki split, binary64 data, n <= 32)
  // Step 1 without its Gram dot products and the T factors' Gram entries on
  // the tensor cores (k_gram_oz): the Ozaki form with a one-row-group tile
  bool gram_oz = false;
  // k_rowmul with two inputs (the adjoint): a register tile close to the
  // b_rm2 rows per block whose two inputs fit in shared memory together
  KernelCfg cfg_rm2;
  int64_t b_rm2 = 0;
  std::vector<Level> levels;  // levels[0] = Step 1; levels[1..] = tree
  size_t off_ctop = 0;   // n x n binary64 top coefficient (sign matrix, or D U_R)
  size_t off_small = 0;  // scratch for small n x n work (SVD, Cholesky, ...)
  size_t bytes = 0;      // workspace of the TSQR-based ops (direct, svd, indirect)
  // Gram-based ops (cholqr, backward): partial Grams + small scratch
  int gram_chunk = 0, gram_grid = 0, gram_nt = 0;
  size_t off_part = 0, off_gsmall = 0, bytes_gram = 0;
};

constexpr int kSmallSlots = 8;  // n x n binary64 matrices in each small scratch area
// Default Step-1 block height.  Small problems: one register tile per block.
// Otherwise the number of blocks is a whole number of waves (CTAs resident
// per SM x SMs), so that no wave runs part-empty, at least kMinWaves blocks
// per SM, with blocks as tall as kMaxTiles tiles allow: tall blocks keep the
// stack of R factors (and so the Step-2 tree) small -- at n = 25 the 608
// R factors of 4 blocks per SM take a two-level tree of 25-way nodes.  The
// flat tree inside a block adds rounding error in proportion to its tiles,
// so double-float compute (unit roundoff 2^-48) takes fewer of them.
constexpr int kMinWaves = 4;
constexpr int kMaxTiles = 64;       // binary64 data
constexpr int kMaxTilesF32 = 128;   // binary32 data: its binary64 tree is costly, its rounding unit large
constexpr int kMaxTilesDF64 = 8;
constexpr int kDefaultSMs = 152;  // GB300
constexpr int kMaxGramParts = 304;  // at most this many partial Grams (2 per SM of a GB300)

// TSQR_PREC_AUTO -> the concrete mode for this dtype and n (other modes
// are returned unchanged): binary32 data at n >= kAutoTf32MinN takes the
// 3xTF32 Step 3 (measured faster than the binary32 FMA Step 3 from about
// n = 16 on; below, the chunk stream's per-chunk cost dominates), binary64
// data at n <= 32 the Ozaki form, everything else the data's own arithmetic.
constexpr int kAutoTf32MinN = 20;
int resolve_prec(int prec, int esz, int64_t n);

// Workspace bytes of `op` (tsqr_op) under a built plan.
size_t op_bytes(const Plan& P, int op);

// Builds the plan; returns 0 or a tsqr_status code.  block_rows > 0 fixes
// the Step-1 block height (any value >= n; above the register tile's B rows
// the block is factored tile by tile); 0 chooses it.
// `sms` = the device's SM count (sizes the default block height).
int make_plan(int64_t m, int64_t n, int esz, int64_t block_rows, int fanout, Plan* plan, int prec = 0,
              int sms = kDefaultSMs);

// Plan of the host-buffer entry point (tsqr_direct_host): the row blocks are
// taken in `chunks` (<= kMaxHostChunks) consecutive groups, each a whole
// number of waves of resident CTAs, so that chunk c's copy overlaps chunk
// c - 1's kernels.  block_rows == 0: the block height is chosen so that A
// splits into chunks of about kHostChunkBytes (at most kMaxHostChunks).
constexpr int kMaxHostChunks = 8;
constexpr int64_t kHostChunkBytes = 128ll << 20;
int make_host_plan(int64_t m, int64_t n, int esz, int64_t block_rows, int fanout, Plan* plan, int* chunks,
                   int prec = 0, int sms = kDefaultSMs);

}  // namespace tsqr
