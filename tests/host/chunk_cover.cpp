// Host check of the Step-3 chunk sequence of chunks.cuh (the streaming
// Step-3 kernels walk it): CTA c of `grid` takes the chunks
// [total c / grid, total (c + 1) / grid), placing its cursor with set() and
// moving it with next(), as the kernel does.  For each geometry read from
// stdin ("m n b B bt grid") it checks that
//   * set(j) and the cursor reached by next() from set(j - 1) agree,
//   * every chunk lies inside its tile, its tile inside its block, its block
//     inside [0, m), with 1 <= rows <= kChunkM and its T slot = blk kt + t,
//   * every row of A is visited exactly once.
// Prints "ok <chunks>" per geometry, or "FAIL <reason>" and exits 1.
#define __device__
#include <cstdio>
#include <vector>

#include "chunks.cuh"

using tsqr::TqCursor;
using tsqr::TqGeom;

static bool same(const TqCursor& a, const TqCursor& b) {
  return a.blk == b.blk && a.rows_b == b.rows_b && a.off == b.off && a.slot == b.slot && a.kt_b == b.kt_b &&
         a.t == b.t && a.cnt == b.cnt && a.c0 == b.c0;
}

int main() {
  long long m, b;
  int n, B, bt, grid;
  while (std::scanf("%lld %d %lld %d %d %d", &m, &n, &b, &B, &bt, &grid) == 6) {
    if (b > m) b = m;
    const int64_t p = (m + b - 1) / b;
    const int kt = static_cast<int>(TqGeom::tiles_of(b, B, bt));  // the plan's tiles per (full) block
    const TqGeom G(m, n, b, B, bt, p);
    const int64_t total = G.total();
    std::vector<unsigned char> seen(static_cast<size_t>(m), 0);
    for (int c = 0; c < grid; ++c) {
      const int64_t lo = total * c / grid, hi = total * (c + 1) / grid;
      TqCursor cur;
      if (lo < hi) cur.set(G, kt, lo);
      for (int64_t j = lo; j < hi; ++j) {
        if (j > lo) {
          cur.next(G, kt);
          TqCursor ref;
          ref.set(G, kt, j);
          if (!same(cur, ref)) { std::printf("FAIL next/set differ at chunk %lld\n", (long long)j); return 1; }
        }
        const int rows = cur.crows();
        if (cur.blk < 0 || cur.blk >= p) { std::printf("FAIL block %lld\n", (long long)cur.blk); return 1; }
        if (cur.off % n != 0) { std::printf("FAIL offset %lld\n", (long long)cur.off); return 1; }
        const int64_t r0 = cur.off / n;
        const int64_t tr0 = cur.t == 0 ? 0 : B + static_cast<int64_t>(cur.t - 1) * bt;
        const int64_t b0 = cur.blk * b;
        if (rows < 1 || rows > tsqr::kChunkM || cur.t < 0 || cur.t >= cur.kt_b || cur.kt_b > kt ||
            r0 < b0 + tr0 + cur.c0 || r0 + rows > b0 + tr0 + cur.cnt || b0 + tr0 + cur.cnt > b0 + cur.rows_b ||
            b0 + cur.rows_b > m || cur.slot != cur.blk * kt + cur.t || cur.slot >= p * kt) {
          std::printf("FAIL chunk %lld: blk %lld t %d c0 %d cnt %d rows %d\n", (long long)j, (long long)cur.blk,
                      cur.t, cur.c0, cur.cnt, rows);
          return 1;
        }
        for (int64_t r = r0; r < r0 + rows; ++r) {
          if (seen[static_cast<size_t>(r)]++) { std::printf("FAIL row %lld twice\n", (long long)r); return 1; }
        }
      }
    }
    for (int64_t r = 0; r < m; ++r)
      if (!seen[static_cast<size_t>(r)]) { std::printf("FAIL row %lld missed\n", (long long)r); return 1; }
    std::printf("ok %lld\n", (long long)total);
  }
  return 0;
}
