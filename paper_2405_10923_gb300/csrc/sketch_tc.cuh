// Gaussian sketch on the tcgen05 tensor cores (sketch_tc.cu).
#pragma once
#include "common.cuh"
#include "sketch.cuh"

namespace rhqr {

// True when the 16-bit Gaussian sketch of an n x m float32 matrix can run on
// the tensor-core kernel (shape and alignment conditions).
bool sketch_tc_supported(const SketchView &s, int64_t n, int32_t m, int32_t c);
size_t sketch_tc_workspace_bytes(const SketchView &s, int64_t n, int32_t m, int32_t c);

// The tensor-core tile order of a 16-bit k x n operator G (row-major, ldg):
// tiles of 256 rows x 64 columns, each 32 KiB laid out as the kernel's shared
// memory holds it (row r at byte 128 r, its 16-byte chunk q at position
// q ^ (r mod 8)), tile (t, b) at byte (t * nkb + b) * 32768 with
// nkb = ceil(n / 64); rows >= k and columns >= n are zero.
size_t operator_tiles_bytes(int64_t n, int32_t k);
int64_t operator_tiles_nkb(int64_t n);
rhqr_status make_operator_tiles(const void *G, int64_t ldg, int64_t n, int32_t k, void *Gt, cudaStream_t st);

// Z = Psi_m X for float32 X (n x c, ldx) with the bf16/f16 Gaussian operator;
// X is split into `limbs` 16-bit terms (1..3).  Every wait of the kernel gives
// up after `budget` polls (<= 0: kDefaultWaitBudget); a wait that ran out
// leaves NaN in the sketch rows of Z and RHQR_ETIMEOUT in info (may be NULL).
rhqr_status sketch_apply_tc(const SketchView &s, int32_t m, const float *X, int64_t n, int32_t c, int64_t ldx,
                            int limbs, double *Z, int64_t ldz, void *ws, size_t ws_bytes, rhqr_info *info,
                            long long budget, cudaStream_t st);

}  // namespace rhqr
