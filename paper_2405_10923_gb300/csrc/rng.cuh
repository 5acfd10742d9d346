// Host entry points of rng.cu.
#pragma once
#include <algorithm>

#include "common.cuh"

namespace rhqr {

uint64_t stream_base(uint64_t seed, uint32_t stream);

// N sign bits (word w, bit b <=> D_{32w+b} = -1) and the k sampled rows.
// scratch: >= 1 KiB + 4 * ceil(N / 1024) bytes of device memory.  Synchronises st.
rhqr_status make_srht_operator(int64_t N, int32_t k, uint64_t seed, uint32_t *sign_bits, int32_t *rows,
                               void *scratch, size_t scratch_bytes, cudaStream_t st);

// G (k x n, row-major, ld = ldg) in `dtype`; coef_scratch: 32 doubles.
rhqr_status make_gaussian_operator(int64_t n, int32_t k, uint64_t seed, int32_t dtype, void *G, int64_t ldg,
                                   double *coef_scratch, cudaStream_t st);

rhqr_status export_signs(const uint32_t *bits, int8_t *out, int64_t N, cudaStream_t st);

}  // namespace rhqr
