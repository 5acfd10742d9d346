// Host entry of the left-looking path (left.cu).
#pragma once
#include "common.cuh"
#include "sketch.cuh"

namespace rhqr {

size_t left_workspace_bytes(const SketchView &s, int64_t n, int32_t m, int32_t wt);

rhqr_status left_factor(const SketchView &s, const void *W, int32_t wt, int64_t n, int32_t m, int64_t ldw,
                        int32_t scaling, void *U, int64_t ldu, double *S, int64_t lds, double *T, double *R, void *Q,
                        int64_t ldq, void *ws, size_t ws_bytes, rhqr_info *info, cudaStream_t st);

// blockRHQR (Algorithm 5) with blocks of bs columns (1 <= bs <= 64); outputs
// as left_factor, with T the compact-form T of all m reflectors (its diagonal
// blocks are the blocks' T^(j)).
size_t block_workspace_bytes(const SketchView &s, int64_t n, int32_t m, int32_t bs, int32_t wt);
rhqr_status block_factor(const SketchView &s, const void *W, int32_t wt, int64_t n, int32_t m, int64_t ldw,
                         int32_t bs, int32_t scaling, void *U, int64_t ldu, double *S, int64_t lds, double *T,
                         double *R, void *Q, int64_t ldq, void *ws, size_t ws_bytes, rhqr_info *info,
                         cudaStream_t st);

// State of one RHQR-Arnoldi process (Algorithm 7): M = mmax + 1 reflectors in
// compact form (U n x M in the basis dtype, S = Psi U, T), Psi = diag(I_M, Omega).
struct ArnoldiState {
  SketchView view;
  int64_t n;
  int32_t M, dtype, scaling, j;
  void *U;
  int64_t ldu;
  double *S;
  int64_t lds;
  double *T, *beta, *gamma, *c, *v, *d, *coef, *y, *z;
  int *stop;
  void *stage;
  size_t stage_bytes;
  void *aws;
  size_t aws_bytes;
};

size_t arnoldi_state_bytes(const SketchView &s, int64_t n, int32_t M, int32_t dt);
rhqr_status arnoldi_carve(ArnoldiState &a, void *mem, size_t bytes);
rhqr_status arnoldi_begin(ArnoldiState &a, const void *r0, double *h0, void *q1, rhqr_info *info, cudaStream_t st);
rhqr_status arnoldi_scale_copy(const ArnoldiState &a, void *Udst, int64_t ldu, cudaStream_t st);
rhqr_status arnoldi_step(ArnoldiState &a, const void *w, double *h, void *qn, rhqr_info *info, cudaStream_t st);
// RHQR-GMRES solution (Algorithm 8): y = argmin ||h0 - H y|| (res = the minimum),
// x = x0 + Q_m y when x != nullptr; scratch holds arnoldi_solution_scratch_doubles(M).
size_t arnoldi_solution_scratch_doubles(int32_t M);
rhqr_status arnoldi_solution(const ArnoldiState &a, double *scratch, const double *H, int64_t ldh, int32_t m,
                             const double *h0, const void *x0, void *x, double *y, double *res, cudaStream_t st);

}  // namespace rhqr
