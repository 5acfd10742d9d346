// Device-side view of a sketch handle and the RHSketch launchers.
#pragma once
#include <algorithm>

#include "common.cuh"

namespace rhqr {

struct SketchView {
  int64_t n, N;
  int32_t k, kind, omega_dtype;
  // SRHT: sign bits, sampled rows and their Kronecker split N = N1 * N2
  const uint32_t *sign_bits;
  const int32_t *rows;
  int32_t N1, N2, d2;          // d2 distinct in-block positions of the sampled rows
  const int32_t *i2_list;      // d2 positions, increasing
  const int32_t *sample_i1;    // k block indices
  const int32_t *sample_slot;  // k slots into i2_list
  // Gaussian: k x n row-major values (ld = ldg) in omega_dtype
  const void *G;
  int64_t ldg;
  // 16-bit Gaussian operators also in tensor-core tile order (sketch_tc.cu):
  // 256 x 64 tiles of 32 KiB, tile (t, b) at byte (t * gt_nkb + b) * 32768
  const void *Gt;
  int64_t gt_nkb;
};

size_t sketch_apply_workspace_bytes(const SketchView &s, int32_t m, int32_t xt, int64_t n, int32_t c);

// One row shard's share of Z = Psi_m X: Z = Psi_m[:, row0:row0+rows] X_local
// (X_local: the global rows row0 .. row0 + rows - 1), so that the shards' Z
// sum to the whole sketch.  SRHT shards start on a segment boundary (row0 a
// multiple of N2).
size_t sketch_rows_workspace_bytes(const SketchView &s, int32_t m, int32_t xt, int64_t row0, int64_t rows,
                                   int32_t c);
rhqr_status sketch_apply_rows_simt(const SketchView &s, int32_t m, const void *X, int32_t xt, int64_t row0,
                                   int64_t rows, int32_t c, int64_t ldx, double *Z, int64_t ldz, void *ws,
                                   size_t ws_bytes, cudaStream_t st);

// Z = Psi_m X with the SIMT kernels (SRHT or Gaussian of any stored dtype).
rhqr_status sketch_apply_simt(const SketchView &s, int32_t m, const void *X, int32_t xt, int64_t n, int32_t c,
                              int64_t ldx, double *Z, int64_t ldz, void *ws, size_t ws_bytes, cudaStream_t st);

}  // namespace rhqr
