// Host launchers of the small FP64 kernels (small.cu).
#pragma once
#include <algorithm>

#include "common.cuh"

namespace rhqr {

size_t hqr_workspace_bytes(int64_t p, int32_t m);
size_t hqr_blocked_workspace_bytes(int64_t p, int32_t m);

// Blocked version (hqr_blocked.cu): RHQR_ENOTSUP when its cluster does not fit.
rhqr_status householder_qr_blocked(const double *Z, int64_t ldz, int64_t p, int32_t m, double *S, int64_t lds,
                                   double *R, double *beta, int32_t scaling, void *ws, size_t ws_bytes,
                                   rhqr_info *info, cudaStream_t st);
rhqr_status copy_f64_2d(const double *A, int64_t lda, int64_t p, int32_t m, double *B, int64_t ldb, cudaStream_t st);

// Householder QR of Z (p x m, ldz): S (p x m, lds), R (m x m), beta (m).
rhqr_status householder_qr_small(const double *Z, int64_t ldz, int64_t p, int32_t m, double *S, int64_t lds,
                                 double *R, double *beta, int32_t scaling, void *ws, size_t ws_bytes,
                                 rhqr_info *info, long long budget, cudaStream_t st);

// T from S and beta (eq. generalwoodburry); SS: m*m doubles of scratch.
rhqr_status t_factor_small(const double *S, int64_t lds, int64_t p, int32_t m, const double *beta, double *SS,
                           double *T, cudaStream_t st);

rhqr_status triu_mul(const double *A, const double *B, int32_t m, double *C, cudaStream_t st);
rhqr_status t_u1t(const double *T, const double *S, int64_t lds, int32_t m, double *Gm, cudaStream_t st);
rhqr_status m_factor(const double *T, const double *S, int64_t lds, const double *Z, int64_t ldz, int64_t p,
                     int32_t m, double *StZ, double *M, cudaStream_t st);
rhqr_status cast_f32(const double *A, int64_t n, float *B, cudaStream_t st);
rhqr_status copy_f64(const double *A, int64_t n, double *B, cudaStream_t st);
rhqr_status info_passes(rhqr_info *info, int32_t passes, cudaStream_t st);
// Column equilibration of a sketch (Z[:, j] /= d_j = ||Z[:, j]||) and the
// column scaling A[:, j] *= d_j that undoes it (on R after the Householder QR,
// on Z itself).
rhqr_status equilibrate_columns(double *Z, int64_t ldz, int64_t p, int32_t m, double *d, cudaStream_t st);
rhqr_status scale_columns(double *A, int64_t lda, int64_t rows, int32_t m, const double *d, cudaStream_t st);

}  // namespace rhqr
