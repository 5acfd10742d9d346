// Gaussian sketch on the tcgen05 tensor cores (sketch_tc.cu).
#pragma once
#include "common.cuh"
#include "sketch.cuh"

namespace rhqr {

// True when the 16-bit Gaussian sketch of an n x m float32 matrix can run on
// the tensor-core kernel (shape and alignment conditions).
bool sketch_tc_supported(const SketchView &s, int64_t n, int32_t m, int32_t c);
size_t sketch_tc_workspace_bytes(const SketchView &s, int64_t n, int32_t m, int32_t c);

// Z = Psi_m X for float32 X (n x c, ldx) with the bf16/f16 Gaussian operator;
// X is split into `limbs` 16-bit terms (1..3).
rhqr_status sketch_apply_tc(const SketchView &s, int32_t m, const float *X, int64_t n, int32_t c, int64_t ldx,
                            int limbs, double *Z, int64_t ldz, void *ws, size_t ws_bytes, cudaStream_t st);

}  // namespace rhqr
