// plan.cpp -- see plan.h.
#include "plan.h"

#include <algorithm>
#include <cstdint>
#include <numeric>

#include "../../include/tsqr.h"
#include "launch.h"
#include "layout.cuh"
#include "oz_kernels.cuh"
#include "tc_kernels.cuh"

namespace tsqr {

static size_t al16(size_t x) { return (x + 15) / 16 * 16; }

// Workspace offsets with overflow checks: *ok is cleared when a sum or
// product does not fit in size_t (only sizes far beyond any device reach it).
static size_t add_ck(size_t a, size_t b, bool* ok) {
  if (a > SIZE_MAX - b) { *ok = false; return 0; }
  return a + b;
}
static size_t mul_ck(size_t a, size_t b, bool* ok) {
  if (b != 0 && a > SIZE_MAX / b) { *ok = false; return 0; }
  return a * b;
}
static size_t al16_ck(size_t x, bool* ok) {
  if (x > SIZE_MAX - 15) { *ok = false; return 0; }
  return al16(x);
}

// Register-tile heights and their thread bounds (must match tiles_f64.h and
// tiles_f32.h).  Each SM sub-partition holds 16K registers
// and a CTA of MAXT threads puts ceil(MAXT/128) warps on each, so the
// per-thread limit is 255 / 168 / 128 / 96 registers at MAXT = 256 / 384 /
// 512 / 640; R x 5 values (x2 registers for 8-byte and double-float values)
// leave about 60 registers for the rest of the kernel, with no spills.
// Tile 4 exceeds that budget (its registers spill); it is taken only when no
// other tile holds the rows asked for (binary64 tree nodes of two R factors
// at n > 64).  Tile 5 is wide: 8 columns per thread, 256 threads (n <= 64),
// taken exactly for 50 < n <= 64, where it beat the 5-column tiles (fewer
// warps sharing each column's reduction and reflector hand-off: 4,000,000 x
// 64 FP64 164.9 -> 114.1 ms, FP32 20.4 -> 18.1 ms); at n <= 50 its padded
// columns and fewer warps make it slower.
struct TileChoice { int R, maxt; bool spills; int npc; };
constexpr int kNumTiles = 7;
static const TileChoice kTiles64[kNumTiles] = {{16, 256, false, kNpc}, {10, 384, false, kNpc}, {6, 512, false, kNpc},
                                               {4, 640, false, kNpc},  {8, 640, true, kNpc},   {12, 256, false, 8},
                                               {5, 384, false, 10}};
static const TileChoice kTiles32[kNumTiles] = {{32, 256, false, kNpc}, {20, 384, false, kNpc}, {12, 512, false, kNpc},
                                               {8, 640, false, kNpc},  {16, 640, true, kNpc},  {24, 256, false, 8},
                                               {10, 384, false, 10}};
// columns per thread preferred for n
static int pref_npc(int n) { return n <= 50 ? kNpc : (n <= 64 ? 8 : 10); }

// Registers a thread may use under __launch_bounds__(maxt, 1): each of the
// 4 sub-partitions holds 16K registers for ceil(maxt / 128) warps.
static int reg_cap(int maxt) {
  const int w = (maxt + 127) / 128;
  int r = 16384 / (32 * w) / 8 * 8;
  return r > 255 ? 255 : r;
}

// Picks the register tile and row-group count.  want_b > 0: the smallest
// capacity B >= want_b (ties: the taller register tile); want_b == 0: the
// default policy below.
bool choose_cfg(int kind, int n, KernelCfg* out, int64_t want_b, int policy, int min_b) {
  if (n < 1 || n > TSQR_NMAX) return false;
  const int esz = kind == kKindF32 ? 4 : 8;
  const TileChoice* tiles = kind == kKindF32 ? kTiles32 : kTiles64;
  KernelCfg best;
  best.kind = kind;
  // pass 0: the tiles of this n's width; pass 1: any spill-free tile;
  // pass 2: the spilling tile.  A wanted capacity (want_b) considers both
  // widths from the start: the tightest fit wins.
  for (int pass = want_b > 0 ? 1 : 0; pass < 3 && best.B == 0; ++pass)
  for (int ti = 0; ti < kNumTiles; ++ti) {
    if (tiles[ti].spills != (pass == 2)) continue;
    if (pass == 0 && tiles[ti].npc != pref_npc(n)) continue;
    const int npc = tiles[ti].npc;
    const int CS = (n + npc - 1) / npc;
    const int NPAD = CS * npc;
    const int R = tiles[ti].R;
    for (int NRG = tiles[ti].maxt / (32 * CS); NRG >= 1; --NRG) {
      const int B = 32 * NRG * R;
      const int NT = 32 * CS * NRG;
      if (B < n || B < min_b) break;
      size_t a = LocalQrSmem(B, n, NT / 32, NPAD, esz, esz).total;
      if (a > kSmemMax) continue;
      int fq_rows = B;  // k_form_q stages its block in chunks of fq_rows rows
      while (fq_rows > 32 && FormQSmem(fq_rows, n, NPAD, esz, esz).total > kSmemMax) fq_rows -= 32;
      size_t f = FormQSmem(fq_rows, n, NPAD, esz, esz).total;
      if (f > kSmemMax) continue;
      int rm_rows = B;  // k_rowmul also stages two n x NPAD matrices: shrink its stage
      while (rm_rows > 32 && RowMulSmem(rm_rows, n, NPAD, esz, esz).total > kSmemMax) rm_rows -= 32;
      if (RowMulSmem(rm_rows, n, NPAD, esz, esz).total > kSmemMax) continue;
      // CTAs of k_local_qr per SM (register cap of the tile, shared memory)
      int ctas = 65536 / (NT * reg_cap(tiles[ti].maxt));
      const int by_smem = (int)(kSmemPerSM / (a + 1024));
      ctas = ctas < by_smem ? ctas : by_smem;
      ctas = ctas < 1 ? 1 : (ctas > 4 ? 4 : ctas);
      bool take;
      if (want_b > 0) {
        take = B >= want_b && (best.B == 0 || B < best.B || (B == best.B && R > best.R));
      } else if (policy == kPolicyLargest) {
        take = B > best.B;  // largest row block wins; ties keep the earlier tile
      } else if (policy == kPolicyInFlight) {
        const int64_t rows = (int64_t)B * ctas, best_rows = (int64_t)best.B * best.ctas;
        take = best.B == 0 || rows > best_rows || (rows == best_rows && ctas > best.ctas);
      } else {
        // Step 1: the largest block (the fixed per-column cost of the
        // Householder loop, and the per-tile cost of blocks of several tiles,
        // are spread over more rows; measured better than two smaller CTAs
        // per SM); ties: fewer threads
        take = best.B == 0 || B > best.B || (B == best.B && NT < best.NT);
      }
      if (take) {
        best.npc = npc; best.R = R; best.CS = CS; best.NRG = NRG; best.NT = NT; best.B = B;
        best.smem_qr = a; best.smem_fq = f; best.tile = ti; best.fq_rows = fq_rows;
        best.rm_rows = rm_rows; best.smem_rm = RowMulSmem(rm_rows, n, NPAD, esz, esz).total;
        best.ctas = ctas;
        // lanes reading one column of consecutive rows (row stride n elements)
        // fall into gcd(n words, 32) banks' worth of conflicts; 8-way or worse
        // is worth the rotated order (which spreads the n x NPAD coefficient
        // reads instead)
        best.skew = std::gcd(n * esz / 4, 32) >= 8 ? 1 : 0;
      }
    }
  }
  if (best.B == 0) return false;
  *out = best;
  return true;
}

GramGeom gram_geom(int64_t m, int n, int esz) {
  GramGeom g;
  int64_t chunk = (int64_t)(kSmemMax - 64) / (2 * (int64_t)n * esz);
  chunk = chunk > 1024 ? 1024 : chunk;
  chunk = chunk / 16 * 16;
  if (chunk < 16) chunk = 16;
  g.chunk = (int)chunk;
  const int64_t nchunks = (m + chunk - 1) / chunk;
  g.grid = (int)(nchunks < kMaxGramParts ? nchunks : kMaxGramParts);
  const int n4 = (n + 3) / 4, n5 = (n + 4) / 5;
  g.tile = (n5 * n5 * 25 < n4 * n4 * 16) ? 5 : 4;  // fewer padded products
  const int nt1 = g.tile == 5 ? n5 : n4;
  int nt = (nt1 * nt1 + 31) / 32 * 32;
  g.nt = nt < 256 ? 256 : (nt > 1024 ? 1024 : nt);
  return g;
}

size_t op_bytes(const Plan& P, int op) {
  return (op == TSQR_OP_CHOLQR || op == TSQR_OP_BACKWARD) ? P.bytes_gram : P.bytes;
}

int resolve_prec(int prec, int esz, int64_t n) {
  if (prec != TSQR_PREC_AUTO) return prec;
  // binary32 data: the Step-3 product on the tensor cores from n = 20 up,
  // where it outruns the FMA form; binary64 data:
  // the error-free (Ozaki) tensor-core products where they apply (n <= 32)
  if (esz == 4) return n >= kAutoTf32MinN ? TSQR_PREC_TF32X3 : TSQR_PREC_NATIVE;
  return n <= kOzMaxN ? TSQR_PREC_OZAKI : TSQR_PREC_NATIVE;
}

int make_plan(int64_t m, int64_t n, int esz, int64_t block_rows, int fanout, Plan* plan, int prec, int sms) {
  if (n < 1 || n > TSQR_NMAX || m < n) return TSQR_ERR_SHAPE;
  // every m x n matrix of the call, at 8 bytes an entry, must have a byte
  // size that int64 holds (the planner and the kernels index with it)
  if (m > INT64_MAX / 8 / n) return TSQR_ERR_SHAPE;
  prec = resolve_prec(prec, esz, n);
  if (prec != TSQR_PREC_NATIVE && !(prec == TSQR_PREC_DF64 && esz == 8) && !(prec == TSQR_PREC_TF32X3 && esz == 4) &&
      !(prec == TSQR_PREC_OZAKI && esz == 8))
    return TSQR_ERR_ARG;
  Plan P;
  P.m = m;
  P.n = n;
  P.esz = esz;
  const int kind0 = esz == 4 ? kKindF32 : (prec == TSQR_PREC_DF64 ? kKindDF64 : kKindF64);
  // Step-1 tile: the most rows resident per SM (double-float: the largest
  // tile); a smaller one when the caller's blocks fit in it
  const int policy0 = kind0 == kKindDF64 ? kPolicyStep1 : kPolicyInFlight;
  if (!choose_cfg(kind0, (int)n, &P.cfg0, 0, policy0) ||
      !choose_cfg(kKindF64, (int)n, &P.cfg64, 0, kPolicyStep1, 2 * (int)n))
    return TSQR_ERR_SHAPE;
  if (block_rows > 0 && block_rows <= P.cfg0.B && !choose_cfg(kind0, (int)n, &P.cfg0, block_rows, kPolicyStep1))
    return TSQR_ERR_SHAPE;
  const int64_t B0 = P.cfg0.B;
  // rows per tile after the first: the register tile less the carried R,
  // rounded down so that every tile starts on a 16-byte boundary when the
  // block does (bulk copies)
  int64_t al = 1;
  while ((al * n * esz) % 16 != 0) ++al;
  const int64_t bt = (B0 - n) / al * al;
  if (bt < 1) return TSQR_ERR_SHAPE;
  int64_t b0 = block_rows;
  if (b0 <= 0) {
    if (sms < 1) sms = kDefaultSMs;
    const int64_t kmax = kind0 == kKindDF64 ? kMaxTilesDF64 : (kind0 == kKindF32 ? kMaxTilesF32 : kMaxTiles);
    const int64_t bmax = B0 + (kmax - 1) * bt;
    if (m <= (int64_t)kMinWaves * sms * P.cfg0.ctas * B0) {
      b0 = B0;
    } else {
      const int64_t slots = (int64_t)sms * P.cfg0.ctas;  // CTAs resident at once
      int64_t waves = (m + slots * bmax - 1) / (slots * bmax);
      const int64_t wmin = (kMinWaves + P.cfg0.ctas - 1) / P.cfg0.ctas;  // kMinWaves blocks per SM
      if (waves < wmin) waves = wmin;
      const int64_t p = waves * slots;
      b0 = (m + p - 1) / p;
      b0 = (b0 + al - 1) / al * al;  // blocks start on 16-byte boundaries
    }
  }
  if (b0 < n) return TSQR_ERR_SHAPE;
  if (b0 > m) b0 = m;  // one block
  const int64_t kt0 = b0 <= B0 ? 1 : 1 + (b0 - B0 + bt - 1) / bt;
  if (kt0 > (1 << 20)) return TSQR_ERR_SHAPE;
  // tree node = f stacked R factors, f >= 2: up to the binary64 row-block
  // tile's rows (fmax), or any f whose node fits one CTA's shared memory or
  // a cluster of f CTAs.  Default: fmax while a node of 4 triangles fits one
  // CTA, else (n > 84, where one CTA holds at most 3) nodes of kTreeClMaxF
  // triangles on clusters: 20,000,000 x 100 has 4 tree levels instead of 10
  const int64_t fmax = P.cfg64.B / n;
  const int ni = static_cast<int>(n);
  const int64_t f = fanout > 0 ? fanout : (fmax >= 4 && tree_up_fits(ni, 4) ? fmax : kTreeClMaxF);
  if (f < 2 || (f > fmax && !tree_up_fits(ni, static_cast<int>(f)) && !tree_up_cl_fits(ni, static_cast<int>(f))))
    return TSQR_ERR_SHAPE;

  P.prec = prec;
  P.tc3 = prec == TSQR_PREC_TF32X3 && n <= kTcwMaxN;
  P.oz3 = prec == TSQR_PREC_OZAKI && n <= kOzMaxN;
  P.gram_oz = P.oz3 && n <= kGmMaxN && P.cfg0.kind == kKindF64 && P.cfg0.NRG == 1;
  {
    const int kind_rm = esz == 4 ? kKindF32 : kKindF64;
    // the coefficient blocks' padded width: the wider of the two tile widths'
    // paddings (the tile chosen below may be either)
    const int NPAD = (int)std::max(std::max((n + kNpc - 1) / kNpc * kNpc, (n + 7) / 8 * 8), (n + 9) / 10 * 10);
    int64_t b2 = 32;
    while (RowMulSmem((int)(2 * (b2 + 32)), (int)n, NPAD, esz, esz).total <= kSmemMax) b2 += 32;
    if (RowMulSmem((int)(2 * b2), (int)n, NPAD, esz, esz).total > kSmemMax) return TSQR_ERR_SHAPE;
    // the smallest tile holding b2 rows, else (small n) the largest tile
    if (!choose_cfg(kind_rm, (int)n, &P.cfg_rm2, b2, kPolicyStep1) &&
        !choose_cfg(kind_rm, (int)n, &P.cfg_rm2, 0, kPolicyLargest))
      return TSQR_ERR_SHAPE;
    P.b_rm2 = P.cfg_rm2.B < b2 ? P.cfg_rm2.B : b2;
    P.cfg_rm2.rm_rows = (int)(2 * P.b_rm2);
    P.cfg_rm2.smem_rm = RowMulSmem(P.cfg_rm2.rm_rows, (int)n, P.cfg_rm2.CS * P.cfg_rm2.npc, esz, esz).total;
  }
  Level l0;
  l0.rows = m;
  l0.b = b0;
  l0.p = (m + b0 - 1) / b0;
  l0.bt = bt;
  l0.kt = (int)kt0;
  P.levels.push_back(l0);
  while (P.levels.back().p > 1) {
    Level l;
    l.rows = P.levels.back().p * n;
    l.b = f * n;
    l.p = (l.rows + l.b - 1) / l.b;
    l.bt = P.cfg64.B - n;  // tree nodes fit one tile (f n <= B)
    l.kt = 1;
    P.levels.push_back(l);
  }
  // The kernels take a block's height as int and launch one CTA per row
  // block, per T slot (the T build) or per triangle of a tree node (cluster
  // nodes): heights and grids beyond int and gridDim.x (2^31 - 1) are shape
  // errors here rather than truncated launch arguments.
  if (b0 > INT32_MAX) return TSQR_ERR_SHAPE;
  for (size_t i = 0; i < P.levels.size(); ++i) {
    const Level& l = P.levels[i];
    if (l.p > INT32_MAX / l.kt || (i > 0 && l.p > INT32_MAX / f)) return TSQR_ERR_SHAPE;
  }
  bool ok = true;
  size_t o = kHeaderBytes;
  const size_t nn = (size_t)n * n * sizeof(double);
  for (auto& l : P.levels) {
    l.off_S = o;
    o = al16_ck(add_ck(o, mul_ck((size_t)l.p, nn, &ok), &ok), &ok);
    l.off_T = o;
    o = al16_ck(add_ck(o, mul_ck(mul_ck((size_t)l.p, (size_t)l.kt, &ok), nn, &ok), &ok), &ok);
  }
  P.off_ctop = o;
  o = al16_ck(add_ck(o, nn, &ok), &ok);
  P.off_small = o;
  o = al16_ck(add_ck(o, kSmallSlots * nn, &ok), &ok);
  P.bytes = o;
  GramGeom g = gram_geom(m, (int)n, esz);
  P.gram_chunk = g.chunk;
  P.gram_grid = g.grid;
  P.gram_nt = g.nt;
  o = kHeaderBytes;
  P.off_part = o;
  o = al16(o + (size_t)g.grid * nn);
  P.off_gsmall = o;
  o = al16(o + kSmallSlots * nn);
  P.bytes_gram = o;
  if (!ok) return TSQR_ERR_SHAPE;
  *plan = P;
  return TSQR_OK;
}

int make_host_plan(int64_t m, int64_t n, int esz, int64_t block_rows, int fanout, Plan* plan, int* chunks,
                   int prec, int sms) {
  Plan P0;
  int rc = make_plan(m, n, esz, block_rows, fanout, &P0, prec, sms);
  if (rc != TSQR_OK) return rc;
  if (sms < 1) sms = kDefaultSMs;
  const int64_t slots = (int64_t)sms * P0.cfg0.ctas;
  if (block_rows <= 0) {
    int64_t c = (m * n * esz) / kHostChunkBytes;
    c = c < 1 ? 1 : (c > kMaxHostChunks ? kMaxHostChunks : c);
    if (c > 1) {
      // c chunks of w waves each, blocks no taller than the default plan's
      const int64_t p0 = P0.levels[0].p;
      const int64_t w = (p0 + c * slots - 1) / (c * slots);
      const int64_t p = c * slots * (w < 1 ? 1 : w);
      int64_t al = 1;
      while ((al * n * esz) % 16 != 0) ++al;
      int64_t b = (m + p - 1) / p;
      b = (b + al - 1) / al * al;
      if (b >= n && b >= P0.cfg0.B) {
        Plan P1;
        if (make_plan(m, n, esz, b, fanout, &P1, prec, sms) == TSQR_OK) P0 = P1;
      }
    }
  }
  const int64_t p = P0.levels[0].p;
  int64_t c = p / slots;
  c = c < 1 ? 1 : (c > kMaxHostChunks ? kMaxHostChunks : c);
  *chunks = (int)c;
  *plan = P0;
  return TSQR_OK;
}

}  // namespace tsqr
