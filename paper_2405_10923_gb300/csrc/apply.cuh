// Host launchers of the row passes (apply.cu).
#pragma once
#include "common.cuh"

namespace rhqr {

int32_t padded_m(int32_t m);
size_t small_padded_bytes(int32_t m);

// out = A (m x m float64, ld m) transposed and padded to mp x mp, cast to T.
template <class T>
rhqr_status pad_transpose(const double *A, int32_t m, int upper, T *out, cudaStream_t st);
template <class T>
rhqr_status pad_transpose_to(const double *A, int32_t m, int32_t mp, int upper, T *out, cudaStream_t st);

// Y[rows] = X[rows] Tri^{-1}  (TriT from pad_transpose with upper = 1)
template <class T>
rhqr_status rows_solve(const T *X, int64_t ldx, int64_t row_begin, int64_t nrows, int32_t m, const T *TriT, T *Y,
                       int64_t ldy, cudaStream_t st);
// U[rows] = X[rows] Tri^{-1} (U may be NULL), Q[rows] = -U[rows] G
template <class T>
rhqr_status rows_solve_mul(const T *X, int64_t ldx, int64_t row_begin, int64_t nrows, int32_t m, const T *TriT,
                           const T *GT, T *U, int64_t ldu, T *Q, int64_t ldq, cudaStream_t st);
// Q[rows] = [I; 0][rows] - U[rows] G
template <class T>
rhqr_status rows_form_q(const T *U, int64_t ldu, int64_t row_begin, int64_t nrows, int32_t m, const T *GT, T *Q,
                        int64_t ldq, cudaStream_t st);
// Q = [I_m; 0] - U G (G upper triangular, m x m float64, overwritten; GT:
// small_padded_bytes(m) of scratch): tensor cores for float32 and m <= 256,
// else the row pass.  A tensor-core wait that ran out is reported in info.
template <class T>
rhqr_status form_q_from_g(const T *U, int64_t ldu, int64_t n, int32_t m, double *Gm, void *GT, T *Q, int64_t ldq,
                          rhqr_info *info, cudaStream_t st);
// U[0:m, :] = S[0:m, :]
template <class T>
rhqr_status top_from_s(const double *S, int64_t lds, int32_t m, T *U, int64_t ldu, cudaStream_t st);

}  // namespace rhqr
