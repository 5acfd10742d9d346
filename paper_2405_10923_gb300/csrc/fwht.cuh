// Unnormalised Walsh-Hadamard transform of one segment of N2 = 2^LOGN2
// entries (512 <= N2 <= 8192) by a block of NT = N2 / 16 threads, in the
// Sylvester order (the SRHT's H, Section 2.3; (H x)_i = sum_j (-1)^popc(i & j) x_j).
//
// Entry e of the segment is written e = r NT + w 32 + l (r < 16 register slot,
// w the warp, l the lane).  Thread (w, l) starts with v[r] = x[r NT + w 32 + l]
// (so every load of the caller is coalesced) and the butterflies run over the
// bits of e in three groups:
//   r bits (4 levels) in registers,
//   l bits (5 levels) by warp shuffles,
//   w bits (LOGN2 - 9 levels) in registers after one transpose through shared
//   memory (thread t then holds the 2^(LOGN2-9) entries that differ only in w).
// Sylvester butterfly on a pair (a at the lower index, b at the upper): a + b
// at the lower, a - b at the upper.  On return buf[e] holds the transform and
// the block is synchronised.
#pragma once
#include <stdint.h>

namespace rhqr {

__device__ __forceinline__ float fwht_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fwht_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <class T, int LOGN2>
__device__ __forceinline__ void fwht_segment(T (&v)[16], T *buf) {
  static_assert(LOGN2 >= 9 && LOGN2 <= 13, "segments of 512 .. 8192 entries");
  constexpr int NT = 1 << (LOGN2 - 4);
  constexpr int WB = LOGN2 - 9;  // warp bits
  const int t = threadIdx.x, lane = t & 31;
  // r bits: entries r and r + h pair up (h = 1, 2, 4, 8)
#pragma unroll
  for (int h = 1; h < 16; h <<= 1)
#pragma unroll
    for (int r = 0; r < 16; ++r)
      if ((r & h) == 0) {
        const T a = v[r], b = v[r + h];
        v[r] = a + b;
        v[r + h] = a - b;
      }
  // lane bits: the upper lane of a pair keeps u - v, the lower v + u, both as
  // one fma(sign, v, u) (exact product by +-1, one rounding: the same value)
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    const T sgn = (lane & s) != 0 ? T(-1) : T(1);
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const T u = __shfl_xor_sync(0xffffffffu, v[r], s);
      v[r] = fwht_fma(sgn, v[r], u);
    }
  }
#pragma unroll
  for (int r = 0; r < 16; ++r) buf[r * NT + t] = v[r];
  __syncthreads();
  if (WB > 0) {
    // thread t takes groups g = t + NT q (g = r 32 + l, q < 16 >> WB) and, in
    // each, the 2^WB entries e = r NT + w 32 + l, w < 2^WB
    constexpr int NW = 1 << WB, NQ = 16 >> WB;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int g = t + NT * q, r = g >> 5, l = g & 31;
      T u[NW];
#pragma unroll
      for (int w = 0; w < NW; ++w) u[w] = buf[r * NT + w * 32 + l];
#pragma unroll
      for (int h = 1; h < NW; h <<= 1)
#pragma unroll
        for (int w = 0; w < NW; ++w)
          if ((w & h) == 0) {
            const T a = u[w], b = u[w + h];
            u[w] = a + b;
            u[w + h] = a - b;
          }
#pragma unroll
      for (int w = 0; w < NW; ++w) buf[r * NT + w * 32 + l] = u[w];
    }
    __syncthreads();
  }
}

}  // namespace rhqr
