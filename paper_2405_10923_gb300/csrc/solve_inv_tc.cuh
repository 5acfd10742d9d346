// Q = X Tri^{-1} as a tensor-core product with the explicit inverse
// (solve_inv_tc.cu), and the FP64 triangular inverse it takes.
#pragma once
#include "common.cuh"

namespace rhqr {

// Rinv = R^{-1} for an upper-triangular m x m float64 R (ld = m), written with
// ld = m (zero below the diagonal).  One warp per column.
rhqr_status upper_inverse(const double *R, int32_t m, double *Rinv, cudaStream_t st);

// True when rows_solve_inv_tc handles m columns.
bool solve_inv_tc_supported(int32_t m);

// Y = X Rinv for float32 X (nrows x m, ldx) and Rinv upper triangular
// (float64, ld = m), Y float32 (ldy).  Y may equal X (in place, same ld).
// With Rinv = D (I + F): A = X D and F split into three bf16 limbs each;
// nprod = 6 takes the six limb products of A F of weight >= 2^-16, nprod = 3
// the three of weight >= 2^-8, nprod = 0 picks 3 when 3 sqrt(m) max|F| <=
// 2^-8 (the dropped products then stay below float32 rounding of Y), else 6.
// A bounded wait that runs out records RHQR_ETIMEOUT in info.
rhqr_status rows_solve_inv_tc(const float *X, int64_t ldx, int64_t nrows, int32_t m, const double *Rinv, int nprod,
                              float *Y, int64_t ldy, rhqr_info *info, long long budget, cudaStream_t st);

}  // namespace rhqr
