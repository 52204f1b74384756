// layout.cuh -- shared-memory layouts of the TSQR kernels, shared by the
// device code and the host planner (which sizes the dynamic shared memory).
#pragma once

#include <cstddef>

#if defined(__CUDACC__)
#define TSQR_HD __host__ __device__
#else
#define TSQR_HD
#endif

namespace tsqr {

TSQR_HD constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Shared-memory layout of k_local_qr (identical on host and device).
struct LocalQrSmem {
  size_t stage, red, xcol, piv, tau, refl, nrm, bar, total;
  TSQR_HD LocalQrSmem(int B, int n, int NW, int NPAD, size_t ssz, size_t tsz) {
    size_t o = 0;
    stage = o; o = align_up(o + (size_t)B * n * ssz, 16);
    // after the register load the stage holds the n x n Gram matrix
    size_t gram_bytes = (size_t)n * n * tsz;
    if ((size_t)B * n * ssz < gram_bytes) o = align_up(stage + gram_bytes, 16);
    red = o; o = align_up(o + 2 * (size_t)NW * 32 * tsz, 16);  // double-buffered partials
    // pivot column: double-buffered (several row groups) or triple-buffered
    // (one row group, where a column's owner may run one column ahead)
    xcol = o; o = align_up(o + 3 * (size_t)B * tsz, 16);
    piv = o; o = align_up(o + 2 * (size_t)NPAD * tsz, 16);    // double-buffered pivot row
    tau = o; o = align_up(o + (size_t)NPAD * tsz, 16);
    refl = o; o = align_up(o + 16 * tsz, 16);                 // reflector scalars, two columns
    nrm = o; o = align_up(o + 2 * 32 * (size_t)tsz, 16);     // look-ahead norms per row group
    bar = o; o = align_up(o + 16, 16);
    total = o;
  }
};

struct FormQSmem {
  size_t stage, xm, wm, bar, total;
  TSQR_HD FormQSmem(int B, int n, int NPAD, size_t ssz, size_t tsz) {
    size_t o = 0;
    stage = o; o = align_up(o + (size_t)B * n * ssz, 16);
    xm = o; o = align_up(o + (size_t)n * NPAD * tsz, 16);
    wm = o; o = align_up(o + (size_t)n * NPAD * tsz, 16);
    bar = o; o = align_up(o + 16, 16);
    total = o;
  }
};

// Shared-memory layout of k_rowmul (one stage; two inputs use its halves).
struct RowMulSmem {
  size_t sx, sy, m1, m2, bar, total;
  TSQR_HD RowMulSmem(int B, int n, int NPAD, size_t ssz, size_t tsz) {
    size_t o = 0;
    sx = o; o = align_up(o + (size_t)B * n * ssz, 16);
    sy = sx;  // when both inputs are present each uses half of the stage
    m1 = o; o = align_up(o + (size_t)n * NPAD * tsz, 16);
    m2 = o; o = align_up(o + (size_t)n * NPAD * tsz, 16);
    bar = o; o = align_up(o + 16, 16);
    total = o;
  }
};

}  // namespace tsqr
