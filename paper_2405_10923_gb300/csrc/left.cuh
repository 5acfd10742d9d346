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

// State of nrhs RHQR-Arnoldi processes (Algorithm 7) sharing one sketch: for
// each, M = mmax + 1 reflectors in compact form (U n x M in the basis dtype,
// S = Psi U, T), Psi = diag(I_M, Omega).  Process b's arrays lie at b times a
// fixed stride: U + b ldu M, S + b lds M, T + b M^2, the M-vectors (beta,
// gamma, c, v, d, coef) + b M, y and z + b (k + M), stop + 4 b.
struct ArnoldiState {
  SketchView view;
  int64_t n;
  int32_t M, dtype, scaling, j, nrhs;
  void *U;
  int64_t ldu;
  double *S;
  int64_t lds;
  double *T, *beta, *gamma, *c, *v, *d, *coef, *y, *z;
  int *stop;
  void *stage;
  int64_t stage_elems;  // per process
  size_t stage_bytes;
  void *aws;
  size_t aws_bytes;
};

size_t arnoldi_state_bytes(const SketchView &s, int64_t n, int32_t M, int32_t dt, int32_t nrhs);
rhqr_status arnoldi_carve(ArnoldiState &a, void *mem, size_t bytes);
// r0, w, q1, qn: n x nrhs (ld n); h0, h: M x nrhs (ld M); info: nrhs records
rhqr_status arnoldi_begin(ArnoldiState &a, const void *r0, double *h0, void *q1, rhqr_info *info, cudaStream_t st);
rhqr_status arnoldi_scale_copy(const ArnoldiState &a, void *Udst, int64_t ldu, cudaStream_t st);
rhqr_status arnoldi_step(ArnoldiState &a, const void *w, double *h, void *qn, rhqr_info *info, cudaStream_t st);
// RHQR-GMRES solution (Algorithm 8) for every process: y = argmin ||h0 - H y||
// (res = the minimum), x = x0 + Q_m y when x != nullptr.  Process b reads H +
// b ldh mmax, h0 + b M, x0 + b n and writes y + b mmax, res + b, x + b n
// (x0 and x in dtype xdt);
// scratch holds arnoldi_solution_scratch_doubles(M, nrhs).
size_t arnoldi_solution_scratch_doubles(int32_t M, int32_t nrhs);
rhqr_status arnoldi_solution(const ArnoldiState &a, double *scratch, const double *H, int64_t ldh, int32_t m,
                             const double *h0, const void *x0, void *x, int32_t xdt, double *y, double *res,
                             cudaStream_t st);

}  // namespace rhqr
