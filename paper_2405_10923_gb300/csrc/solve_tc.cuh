// Tensor-core row-wise triangular solve (solve_tc.cu).
#pragma once
#include "common.cuh"

namespace rhqr {

// Panel width of the tensor-core solve: Tri must be padded to a multiple.
constexpr int32_t kSolvePanel = 64;

bool solve_tc_supported(int32_t m);

// Y[rows] = X[rows] Tri^{-1} for float32 X, Tri upper triangular given as
// TriT (mp x mp float32, row-major, identity-padded, mp >= ceil(m/64)*64).
// Every wait gives up after `budget` polls (<= 0: kDefaultWaitBudget) and
// records RHQR_ETIMEOUT in info (may be NULL).
rhqr_status rows_solve_tc(const float *X, int64_t ldx, int64_t row_begin, int64_t nrows, int32_t m,
                          const float *TriT, int32_t mp_tri, float *Y, int64_t ldy, rhqr_info *info, long long budget,
                          cudaStream_t st);

}  // namespace rhqr
