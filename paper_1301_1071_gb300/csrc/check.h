// check.h -- geometry and launcher of the compensated accuracy check
// (tsqr_accuracy; check.cu).  Host code.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace tsqr {

// rows x n binary64 values staged per chunk (two matrices): at most
// 2 x 6,144 values, plus R, within one CTA's shared memory
constexpr int64_t kAccuracySmemRows = 6144;
constexpr int kAccuracyMaxParts = 304;  // partial sums (CTAs): 2 per SM of a GB300

struct AccuracyGeom {
  int ch = 0;           // rows per staged chunk
  int grid = 0;         // CTAs = partial sums
  size_t part_bytes = 0;
  size_t smem = 0;
};

AccuracyGeom accuracy_geom(int64_t m, int n);

// out (3 n^2 + 2 binary64, device): hi and lo of Q^T Q - I, E^T E of the
// residual E = A - Q R, ||E||_F^2, ||A||_F^2 (the residual parts zero when
// A is NULL).  part: accuracy_geom(m, n).part_bytes of device scratch.
cudaError_t launch_accuracy(int esz, const void* Q, const void* A, const double* R, int64_t m, int n,
                            double* part, double* out, cudaStream_t st);

}  // namespace tsqr
