// Tensor-core row-wise triangular solve (solve_tc.cu).
#pragma once
#include "common.cuh"

namespace rhqr {

// Panel width of the tensor-core solve: Tri must be padded to a multiple.
constexpr int32_t kSolvePanel = 64;

bool solve_tc_supported(int32_t m);

// Y[rows] = X[rows] Tri^{-1} for float32 X, Tri upper triangular given as
// TriT (mp x mp float32, row-major, identity-padded, mp >= ceil(m/64)*64).
// err: one int of device scratch (bounded-wait timeout flag).
rhqr_status rows_solve_tc(const float *X, int64_t ldx, int64_t row_begin, int64_t nrows, int32_t m,
                          const float *TriT, int32_t mp_tri, float *Y, int64_t ldy, int *err, cudaStream_t st);

}  // namespace rhqr
