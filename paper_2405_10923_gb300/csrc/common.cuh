// Shared definitions of the CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <utility>

#include "../../include/rhqr.h"

namespace rhqr {

// Launch/runtime error -> RHQR_ECUDA (synchronous part of the contract); the
// CUDA error code is kept for rhqr_last_cuda_error.
void note_cuda_error(cudaError_t e);
#define RHQR_CUDA_TRY(expr)                                    \
  do {                                                         \
    cudaError_t e_ = (expr);                                   \
    if (e_ != cudaSuccess) {                                   \
      ::rhqr::note_cuda_error(e_);                             \
      (void)cudaGetLastError();                                \
      return RHQR_ECUDA;                                       \
    }                                                          \
  } while (0)

#define RHQR_TRY(expr)                 \
  do {                                 \
    rhqr_status s_ = (expr);           \
    if (s_ != RHQR_OK) return s_;      \
  } while (0)

// Launch counter (read through rhqr_launch_count): every kernel launch of the
// library is followed by RHQR_LAUNCH_CHECK, which counts it.
void count_launch();
#define RHQR_LAUNCH_CHECK()            \
  do {                                 \
    ::rhqr::count_launch();            \
    RHQR_CUDA_TRY(cudaGetLastError()); \
  } while (0)

// Phase timing with CUDA events on the launching stream (rhqr_profile_*).
enum Phase { PH_SKETCH = 0, PH_HQR, PH_TFACTOR, PH_SOLVE, PH_SMALL, PH_LEFT_STEP, PH_COUNT };
struct PhaseScope {
  int phase;
  cudaStream_t st;
  void *ev;
  PhaseScope(int ph, cudaStream_t s);
  ~PhaseScope();
};

// Polls of a device-side wait before it gives up with RHQR_ETIMEOUT, unless
// the caller sets rhqr_opts.wait_budget.
constexpr long long kDefaultWaitBudget = 20000000LL;

// Programmatic dependent launch (PDL).  A kernel launched with launch_pdl may
// be scheduled before the previous kernel of its stream has finished; it must
// call pdl_wait() before it touches anything that kernel writes (the wait
// returns at once for a kernel launched without PDL).  pdl_release() lets the
// next PDL kernel of the stream be scheduled now; its pdl_wait() still waits
// for this kernel to complete and its writes to be visible.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

inline size_t dtype_size(int32_t t) {
  switch (t) {
    case RHQR_F64: return 8;
    case RHQR_F32: return 4;
    case RHQR_BF16:
    case RHQR_F16: return 2;
    default: return 0;
  }
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Bump allocator over a caller-provided workspace.
struct Carver {
  char *base;
  size_t cap, off;
  Carver(void *p, size_t c) : base((char *)p), cap(c), off(0) {}
  template <class T>
  T *take(size_t count) {
    off = align_up(off, 256);
    size_t bytes = count * sizeof(T);
    if (base == nullptr) {  // sizing pass
      off += bytes;
      return nullptr;
    }
    if (off + bytes > cap) {
      off = cap + 1;
      return nullptr;
    }
    T *p = (T *)(base + off);
    off += bytes;
    return p;
  }
  bool overflow() const { return base != nullptr && off > cap; }
  size_t used() const { return off; }
};

// ----------------------------------------------------------------------------
// device helpers
// ----------------------------------------------------------------------------

template <class T>
__device__ __forceinline__ double to_f64(T v);
template <>
__device__ __forceinline__ double to_f64<double>(double v) { return v; }
template <>
__device__ __forceinline__ double to_f64<float>(float v) { return (double)v; }

template <>
__device__ __forceinline__ double to_f64<__nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
template <>
__device__ __forceinline__ double to_f64<__half>(__half v) { return (double)__half2float(v); }

template <class T>
__device__ __forceinline__ T from_f64(double v);
template <>
__device__ __forceinline__ double from_f64<double>(double v) { return v; }
template <>
__device__ __forceinline__ float from_f64<float>(double v) { return (float)v; }

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (fixed order: lane tree, then warp tree).  `red` holds >= 32
// doubles of shared memory.  Every thread gets the result.
__device__ __forceinline__ double block_sum(double v, double *red) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < (unsigned)nw) ? red[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

// Record a device-side condition in the caller's info (first writer wins).
__device__ __forceinline__ void set_status(rhqr_info *info, int32_t st, int32_t col) {
  if (info == nullptr) return;
  if (atomicCAS(&info->status, (int)RHQR_OK, st) == RHQR_OK) info->column = col;
}

// Backward column sweep of an upper-triangular recurrence, one column per warp
// (m <= 256; lane q owns rows q, q + 32, ...):
//   x_j = top;  for l = j, ..., 1:  s_i += M[i, l] x_l (i < l),  x_{l-1} = f(l-1) s_{l-1}
// with M column-major (M[i, l] at M[l * ldm + i]) and f(i) = -fin[i] (or, with
// fin_recip_diag, -1 / M[i, i]).  Columns of M are fetched DEPTH steps ahead.
// Writes x_i (i <= j) and 0 (j < i < m) to out[0 .. m).
template <int DEPTH>
__device__ __forceinline__ void column_sweep(const double *M, int64_t ldm, int32_t m, int j, double top,
                                             const double *fin, bool fin_recip_diag, double *out) {
  constexpr int PER = 8;
  const int lane = threadIdx.x & 31;
  double s[PER], x[PER], f[PER], buf[DEPTH][PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = lane + 32 * q;
    s[q] = 0.0;
    x[q] = 0.0;
    f[q] = i < j ? (fin_recip_diag ? -1.0 / M[(int64_t)i * ldm + i] : -fin[i]) : 0.0;
  }
#pragma unroll
  for (int d = 0; d < DEPTH; ++d)
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int l = j - d, i = lane + 32 * q;
      buf[d][q] = (l >= 1 && i < l) ? M[(int64_t)l * ldm + i] : 0.0;
    }
  double xl = top;
  int l = j;
  while (l >= 1) {
#pragma unroll
    for (int d = 0; d < DEPTH; ++d) {
      if (l >= 1) {
        double cand = 0.0;
        const int qa = (l + 31) >> 5;  // row groups with rows < l (warp-uniform)
#pragma unroll
        for (int q = 0; q < PER; ++q) {
          if (q < qa) {
            const int i = lane + 32 * q;
            if (i == l) x[q] = xl;
            if (i < l) s[q] += buf[d][q] * xl;
            if (i == l - 1) cand = f[q] * s[q];
          } else if (lane + 32 * q == l) {
            x[q] = xl;
          }
        }
        // refill this slot with column l - DEPTH
#pragma unroll
        for (int q = 0; q < PER; ++q) {
          const int ln = l - DEPTH, i = lane + 32 * q;
          buf[d][q] = (ln >= 1 && i < ln) ? M[(int64_t)ln * ldm + i] : 0.0;
        }
        xl = __shfl_sync(0xffffffffu, cand, (l - 1) & 31);
        --l;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int i = lane + 32 * q;
    if (i == 0) x[q] = xl;
    if (i < m) out[i] = i <= j ? x[q] : 0.0;
  }
}

// Grid-wide barrier for cooperative launches, with a bounded wait.
// `bar[0]` counts arrivals, `bar[1]` is the generation.  Returns false (and
// records RHQR_ETIMEOUT) if the wait ran out; every block then stops.
__device__ __forceinline__ bool grid_barrier(unsigned int *bar, long long budget, rhqr_info *info,
                                             volatile int *abort_flag) {
  __syncthreads();
  __shared__ int ok_s;
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int *vgen = bar + 1;
    unsigned int gen = *vgen;
    __threadfence();
    unsigned int arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (*vgen == gen) {
        if (*abort_flag) { ok = 0; break; }
        if (++it > budget) {
          ok = 0;
          *abort_flag = 1;
          set_status(info, RHQR_ETIMEOUT, -1);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

}  // namespace rhqr
