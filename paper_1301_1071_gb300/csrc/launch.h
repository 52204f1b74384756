// launch.h -- host launchers of the TSQR kernels (internal, C++ linkage).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "plan.h"

namespace tsqr {

// Step 1 / tree level: p CTAs, one per row block of b rows (k.kind selects
// the storage/compute types).
// Blocks of b rows; a block taller than the register tile (b > k.B) is
// factored as tiles of k.B rows and then bt rows, kt tiles at most
// (T slots per block).
cudaError_t launch_local_qr(const KernelCfg& k, const void* A, int64_t m, int n, int64_t b, int64_t bt, int kt,
                            int64_t p, void* Y, double* Rst, double* Tst, int32_t* status, cudaStream_t st);
// Step 3 / tree down-pass: p CTAs.
cudaError_t launch_form_q(const KernelCfg& k, const void* Y, int64_t m, int n, int64_t b, int64_t bt, int kt,
                          int64_t p, const double* T, const double* C, int64_t cblocks, void* Q,
                          int32_t* status, cudaStream_t st);

// Step-2 up pass of one tree level (binary64): node b = f stacked
// triangular blocks of X (rows x n) -> its R (raw signs) into Rout's block
// b; with Y (may alias X): the Householder vectors over the node's rows and
// tau + Gram entries into the node's T slot (Tst); Y == NULL: R only.
// tree_up_fits: the node fits one CTA's shared memory.  tree_up_cl_fits:
// the node fits a cluster of f CTAs, one block each (launch_tree_up_cl, same
// outputs).  Neither: the row-block kernel takes the level.
constexpr int kTreeClMaxF = 8;  // portable cluster size
bool tree_up_fits(int n, int f);
cudaError_t launch_tree_up(const double* X, int64_t rows, int n, int f, int64_t p, double* Y, double* Rout,
                           double* Tst, cudaStream_t st);
bool tree_up_cl_fits(int n, int f);
cudaError_t launch_tree_up_cl(const double* X, int64_t rows, int n, int f, int64_t p, double* Y, double* Rout,
                              double* Tst, cudaStream_t st);

// Step-2 down pass of one tree level (binary64): node b's rows of Y (f
// stacked blocks of n rows, the last node possibly fewer) become its
// children's coefficient blocks from C (cblocks == 1: one block for all),
// using Y = [I; V_2; ...; V_f] with V_k upper triangular.
cudaError_t launch_tree_down(double* Y, int64_t rows, int n, int f, int64_t p, const double* T, const double* C,
                             int64_t cblocks, cudaStream_t st);

// Step 3 for binary32 data on the tensor cores (3xTF32), n <= 100; the block
// and tile geometry (b, B = the Step-1 register tile, bt, kt) of Step 1.  For
// n <= 64 the T slots and C are overwritten (with W and X_0).
cudaError_t launch_form_q_tc(float* Y, int64_t m, int n, int64_t b, int B, int64_t bt, int kt, int64_t p,
                             double* T, double* C, int64_t cblocks, int32_t* status, cudaStream_t st);

// Step 3 for binary64 data with the product Y W on the tensor cores by
// Ozaki splitting (binary16 digits, exact binary32 accumulation), n <= 32;
// the block and tile geometry of Step 1.
cudaError_t launch_form_q_oz(double* Y, int64_t m, int n, int64_t b, int B, int64_t bt, int kt, int64_t p,
                             const double* T, const double* C, int64_t cblocks, int32_t* status, cudaStream_t st);

// The Gram entries v_i^T v_c (i < c) of every tile's Householder vectors
// into the T slots' strictly upper triangles (binary64 data, n <= 32), on the
// tensor cores by Ozaki splitting; Step 1 ran without its Gram dot products
// (launch_local_qr_nogram_f64, which writes Y, R and tau).
cudaError_t launch_gram_oz(const double* Y, int64_t m, int n, int64_t b, int B, int64_t bt, int kt, int64_t p,
                           double* T, int32_t* status, cudaStream_t st);

// out_r = X_r M1 + Y_r M2 over p blocks of b rows (X or Y may be NULL).
cudaError_t launch_rowmul(const KernelCfg& k, const void* X, const double* M1, const void* Y,
                          const double* M2, int64_t m, int n, int64_t b, int64_t p, void* out, int32_t* status,
                          cudaStream_t st);
// Partial Grams X^T Y (grid partials of n x n binary64), then their fixed-order sum into G.
// acc_storage: per-CTA partial Grams accumulate in the storage type (binary32
// data: the FMA pipe); the cross-CTA sum is always binary64.
cudaError_t launch_gram(int esz, const void* X, const void* Y, int64_t m, int n, double* part, double* G,
                        int32_t* status, cudaStream_t st, bool acc_storage = false);

// Gram launch geometry shared by the planner and the launcher.
struct GramGeom { int chunk, grid, nt, tile; };
GramGeom gram_geom(int64_t m, int n, int esz);

}  // namespace tsqr
