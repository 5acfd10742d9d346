// Left-looking trimRHQR (trim.cu).
#pragma once
#include "common.cuh"
#include "sketch.cuh"

namespace rhqr {

size_t trim_workspace_bytes(const SketchView &s, int64_t n, int32_t m, int32_t wt);

// Outputs: U (n x m), S = Omega' U (k x m, lds >= k), T and Tt (m x m, ld m),
// R (m x m), Q (n x m, optional).
rhqr_status trim_factor(const SketchView &s, const void *W, int32_t wt, int64_t n, int32_t m, int64_t ldw,
                        int32_t scaling, void *U, int64_t ldu, double *S, int64_t lds, double *T, double *Tt,
                        double *R, void *Q, int64_t ldq, void *ws, size_t ws_bytes, rhqr_info *info,
                        cudaStream_t st);

}  // namespace rhqr
