// chunks.cuh -- the chunk sequence of the streaming Step-3 kernels
// (k_form_q_tc): the rows of every tile of every row block in
// pieces of kChunkM rows, walked block by block, tile by tile.  Device code
// except the geometry (which the launchers use for the grid).
#pragma once

#include <cstdint>

#include "layout.cuh"

namespace tsqr {

constexpr int kChunkM = 128;  // rows per chunk (tensor-memory lanes)

// The chunks of Step 3: tile t of a block of `rows` rows holds rows
// [0, min(rows, B)) (t = 0) or [B + (t-1) bt, ..) (at most bt rows); each
// tile is cut into chunks of kChunkM rows, taken block by block, tile by tile.
struct TqGeom {
  int64_t m, b, p;
  int n, B, bt;
  int64_t cpb_full, cpb_last, nfull;  // chunks per full block, of the last block; chunks of the full blocks
  TSQR_HD static int64_t tiles_of(int64_t rows, int B, int bt) { return rows <= B ? 1 : 1 + (rows - B + bt - 1) / bt; }
  TSQR_HD static int64_t chunks_of(int64_t rows, int B, int bt) {
    const int64_t r0 = rows < B ? rows : B;
    int64_t c = (r0 + kChunkM - 1) / kChunkM;
    if (rows > B) {
      const int64_t kt = tiles_of(rows, B, bt);
      const int64_t last = rows - B - (kt - 2) * bt;
      c += (kt - 2) * ((bt + kChunkM - 1) / kChunkM) + (last + kChunkM - 1) / kChunkM;
    }
    return c;
  }
  TSQR_HD TqGeom(int64_t m_, int n_, int64_t b_, int B_, int bt_, int64_t p_)
      : m(m_), b(b_), p(p_), n(n_), B(B_), bt(bt_) {
    cpb_full = chunks_of(b, B, bt);
    cpb_last = chunks_of(m - (p - 1) * b, B, bt);
    nfull = (p - 1) * cpb_full;
  }
  TSQR_HD int64_t total() const { return nfull + cpb_last; }
  TSQR_HD int64_t rows_of(int64_t blk) const { return blk == p - 1 ? m - (p - 1) * b : b; }
};

// A position in the chunk sequence: set() places it (divisions), next()
// moves it one chunk on (no division but at a block change).
struct TqCursor {
  int64_t blk, rows_b;  // block and its rows
  int64_t off;          // element offset of the chunk in Y (its first row times n)
  int64_t slot;         // T slot of the chunk's tile (blk kt + t)
  int kt_b, t, cnt, c0;  // tiles of the block, tile, its rows, chunk offset in the tile
  __device__ void tile(const TqGeom& G, int kt) {
    const int64_t tr0 = t == 0 ? 0 : G.B + static_cast<int64_t>(t - 1) * G.bt;
    const int64_t left = rows_b - tr0;
    cnt = static_cast<int>(t == 0 ? (rows_b < G.B ? rows_b : G.B) : (left < G.bt ? left : G.bt));
    off = (blk * G.b + tr0 + c0) * G.n;
    slot = blk * kt + t;
  }
  __device__ void block(const TqGeom& G) {
    rows_b = G.rows_of(blk);
    kt_b = static_cast<int>(TqGeom::tiles_of(rows_b, G.B, G.bt));
  }
  __device__ void set(const TqGeom& G, int kt, int64_t j) {
    int64_t jj;
    if (j < G.nfull) {
      blk = j / G.cpb_full;
      jj = j - blk * G.cpb_full;
    } else {
      blk = G.p - 1;
      jj = j - G.nfull;
    }
    block(G);
    const int64_t r0 = rows_b < G.B ? rows_b : G.B;
    const int64_t ch0 = (r0 + kChunkM - 1) / kChunkM, chb = (G.bt + kChunkM - 1) / kChunkM;
    if (jj < ch0) {
      t = 0;
      c0 = static_cast<int>(jj) * kChunkM;
    } else {
      t = 1 + static_cast<int>((jj - ch0) / chb);
      c0 = static_cast<int>((jj - ch0) % chb) * kChunkM;
    }
    tile(G, kt);
  }
  __device__ void next(const TqGeom& G, int kt) {
    c0 += kChunkM;
    off += static_cast<int64_t>(kChunkM) * G.n;
    if (c0 >= cnt) {
      c0 = 0;
      if (++t >= kt_b) {
        t = 0;
        if (++blk < G.p) block(G);
      }
      if (blk < G.p) tile(G, kt);
    }
  }
  __device__ int crows() const { return cnt - c0 < kChunkM ? cnt - c0 : kChunkM; }
  __device__ int ntop(int n) const { return (t == 0 && c0 == 0) ? static_cast<int>(rows_b < n ? rows_b : n) : 0; }
};

}  // namespace tsqr
