// Column kernels shared by the left-looking family (left.cu: Algorithm 4,
// blockRHQR, RHQR-Arnoldi; trim.cu: left-looking trimRHQR): the refresh of
// one column with earlier reflectors (w <- w - U c, with the deferred scaling
// of the newest reflector), fused with or followed by its sketch.
#pragma once
#include <algorithm>

#include "common.cuh"
#include "fwht.cuh"
#include "sketch.cuh"

namespace rhqr {

// ---------------------------------------------------------------------------
// step 2: column kernels
// ---------------------------------------------------------------------------
// Element strides between the problems of a batch of same-shape independent
// problems (the RHQR-Arnoldi processes of several right-hand sides): a kernel
// launched with gridDim.y = batch count works on problem blockIdx.y.  All zero
// for a single problem.
struct Batch {
  int64_t W, U;      // input column(s), reflector matrix (elements of the data type)
  int64_t vec;       // per-problem vectors of length M (coefficients, gamma, beta, ...)
  int64_t y;         // sketch vectors
  int64_t stage;     // transform / partial-product staging
};

struct ColArgs {
  const void *W;
  int64_t ldw;
  void *U;
  int64_t ldu;
  int64_t n;
  int32_t m, j;
  const double *c;      // j coefficients
  const double *gamma;  // gamma[j-1] scales column j-1
  double *y;            // (k+m) sketch, rows < m written here
  int32_t unit;         // unit-diagonal scaling: u_jj = 1 exactly
  int32_t lo;           // first column of the block whose reflectors refresh column j (0: all)
  int32_t skm;          // leading rows left out of the sketch: m for Psi_m = diag(I_m, Omega), 0 for Omega_full
  Batch bt;             // batch strides (zero for one problem)
};

// The arguments of problem blockIdx.y of a batch.
template <class T>
__device__ __forceinline__ ColArgs batch_args(const ColArgs &a0) {
  ColArgs a = a0;
  const int64_t b = blockIdx.y;
  a.W = (const T *)a0.W + b * a0.bt.W;
  a.U = (T *)a0.U + b * a0.bt.U;
  a.c = a0.c + b * a0.bt.vec;
  a.gamma = a0.gamma + b * a0.bt.vec;
  a.y = a0.y + b * a0.bt.y;
  return a;
}

template <class T>
__device__ __forceinline__ T refresh_row(const ColArgs &a, int64_t i, const double *c_s, T inv_g) {
  const T *W = (const T *)a.W;
  T *U = (T *)a.U;
  T w = W[(int64_t)a.j * a.ldw + i];
  const int j = a.j, lo = a.lo;
  // previous columns of the block, the last one still unscaled
  for (int l = lo; l + 1 < j; ++l) w -= U[(int64_t)l * a.ldu + i] * (T)c_s[l - lo];
  if (j - 1 >= lo) {
    T *up = U + (int64_t)(j - 1) * a.ldu + i;
    T u = (i < j - 1) ? T(0) : ((i == j - 1 && a.unit) ? T(1) : *up * inv_g);
    *up = u;
    w -= u * (T)c_s[j - 1 - lo];
  }
  U[(int64_t)j * a.ldu + i] = w;
  return w;
}

// Refresh of column j over all rows with the whole GPU (one row per thread,
// grid-stride): w_j <- w_j - U_{j-1} c (the previous columns read with four
// independent partial sums), the deferred scaling of column j-1, and the exact
// top rows of the sketch.
template <class T>
__global__ void __launch_bounds__(256) left_refresh_kernel(ColArgs a0) {
  pdl_wait();  // the refresh's coefficients come from the previous kernel
  const ColArgs a = batch_args<T>(a0);
  __shared__ T c_s[1024];  // coefficients, converted once
  const int j = a.j, lo = a.lo, nc = j - lo;
  for (int l = threadIdx.x; l < nc; l += blockDim.x) c_s[l] = (T)a.c[l];
  const T inv_g = (j - 1 >= lo) ? (T)(1.0 / a.gamma[j - 1]) : T(1);
  __syncthreads();
  const T *W = (const T *)a.W;
  T *U = (T *)a.U;
  const int64_t ldu = a.ldu;
  // the fully scaled columns lo .. j-2 with eight independent loads and
  // partial sums in flight per thread; column j-1 (deferred scale) last
  const int nfull = nc > 0 ? nc - 1 : 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    T p[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) p[q] = T(0);
    const T *up = U + (int64_t)lo * ldu + i;
    int l = 0;
    for (; l + 8 <= nfull; l += 8) {
#pragma unroll
      for (int q = 0; q < 8; ++q) p[q] += up[q * ldu] * c_s[l + q];
      up += 8 * ldu;
    }
    for (; l < nfull; ++l, up += ldu) p[l & 7] += *up * c_s[l];
    T w = W[(int64_t)j * a.ldw + i] - (((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7])));
    if (j - 1 >= lo) {
      T *ul = U + (int64_t)(j - 1) * ldu + i;
      const T u = (i < j - 1) ? T(0) : ((i == j - 1 && a.unit) ? T(1) : *ul * inv_g);
      *ul = u;
      w -= u * c_s[nc - 1];
    }
    U[(int64_t)j * ldu + i] = w;
    if (i < a.m) a.y[i] = (double)w;
  }
}

// Vector form of the refresh for 16-byte aligned columns (ldw, ldu multiples
// of 16 bytes, aligned bases): each thread takes V = 16 / sizeof(T)
// consecutive rows with one 16-byte load per column; rows past the last full
// vector go through the scalar loop of the first thread of the grid.
template <class T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int V = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int V = 2;
};

template <class T>
__global__ void __launch_bounds__(256) left_refresh_vec_kernel(ColArgs a0) {
  pdl_wait();  // the refresh's coefficients come from the previous kernel
  using VT = typename Vec16<T>::type;
  constexpr int V = Vec16<T>::V;
  const ColArgs a = batch_args<T>(a0);
  __shared__ T c_s[1024];
  const int j = a.j, lo = a.lo, nc = j - lo;
  for (int l = threadIdx.x; l < nc; l += blockDim.x) c_s[l] = (T)a.c[l];
  const T inv_g = (j - 1 >= lo) ? (T)(1.0 / a.gamma[j - 1]) : T(1);
  __syncthreads();
  const T *W = (const T *)a.W;
  T *U = (T *)a.U;
  const int64_t ldu = a.ldu;
  const int nfull = nc > 0 ? nc - 1 : 0;
  const int64_t nvec = a.n / V;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nvec + (a.n % V != 0);
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = q * V;
    T w[V];
    if (q < nvec) {
      T p[4][V];
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int e = 0; e < V; ++e) p[t][e] = T(0);
      const T *up = U + (int64_t)lo * ldu + i0;
      int l = 0;
      for (; l + 4 <= nfull; l += 4) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const VT u = *reinterpret_cast<const VT *>(up + t * ldu);
          const T *ue = reinterpret_cast<const T *>(&u);
#pragma unroll
          for (int e = 0; e < V; ++e) p[t][e] += ue[e] * c_s[l + t];
        }
        up += 4 * ldu;
      }
      for (; l < nfull; ++l, up += ldu) {
        const VT u = *reinterpret_cast<const VT *>(up);
        const T *ue = reinterpret_cast<const T *>(&u);
#pragma unroll
        for (int e = 0; e < V; ++e) p[l & 3][e] += ue[e] * c_s[l];
      }
      const VT wv = *reinterpret_cast<const VT *>(W + (int64_t)j * a.ldw + i0);
      const T *we = reinterpret_cast<const T *>(&wv);
#pragma unroll
      for (int e = 0; e < V; ++e) w[e] = we[e] - ((p[0][e] + p[1][e]) + (p[2][e] + p[3][e]));
      if (j - 1 >= lo) {
        T *ul = U + (int64_t)(j - 1) * ldu + i0;
        VT uv = *reinterpret_cast<const VT *>(ul);
        T *ue = reinterpret_cast<T *>(&uv);
#pragma unroll
        for (int e = 0; e < V; ++e) {
          const int64_t i = i0 + e;
          const T u = (i < j - 1) ? T(0) : ((i == j - 1 && a.unit) ? T(1) : ue[e] * inv_g);
          ue[e] = u;
          w[e] -= u * c_s[nc - 1];
        }
        *reinterpret_cast<VT *>(ul) = uv;
      }
      VT out;
      T *oe = reinterpret_cast<T *>(&out);
#pragma unroll
      for (int e = 0; e < V; ++e) oe[e] = w[e];
      *reinterpret_cast<VT *>(U + (int64_t)j * ldu + i0) = out;
#pragma unroll
      for (int e = 0; e < V; ++e)
        if (i0 + e < a.m) a.y[i0 + e] = (double)w[e];
    } else {
      // the last n % V rows, one at a time (the same arithmetic as refresh_row)
      for (int64_t i = i0; i < a.n; ++i) {
        T ps[4] = {T(0), T(0), T(0), T(0)};
        for (int l = 0; l < nfull; ++l) ps[l & 3] += U[(int64_t)(lo + l) * ldu + i] * c_s[l];
        T wi = W[(int64_t)j * a.ldw + i] - ((ps[0] + ps[1]) + (ps[2] + ps[3]));
        if (j - 1 >= lo) {
          T *ul = U + (int64_t)(j - 1) * ldu + i;
          const T u = (i < j - 1) ? T(0) : ((i == j - 1 && a.unit) ? T(1) : *ul * inv_g);
          *ul = u;
          wi -= u * c_s[nc - 1];
        }
        U[(int64_t)j * ldu + i] = wi;
        if (i < a.m) a.y[i] = (double)wi;
      }
    }
  }
}

// The refresh of column j (nprob problems of a batch) with the whole GPU: the
// vector kernel when every column start is 16-byte aligned, else the scalar one.
template <class T>
static rhqr_status launch_refresh(const ColArgs &ca, unsigned nprob, cudaStream_t st) {
  constexpr int V = Vec16<T>::V;
  const bool aligned = ca.ldw % V == 0 && ca.ldu % V == 0 && ((uintptr_t)ca.W % 16) == 0 &&
                       ((uintptr_t)ca.U % 16) == 0 && (nprob == 1 || (ca.bt.W % V == 0 && ca.bt.U % V == 0));
  const int64_t units = aligned ? ceil_div(ca.n, V) : ca.n;
  const dim3 g((unsigned)std::min<int64_t>(ceil_div(units, 256), std::max<int64_t>(1, 152 * 8 / (int64_t)nprob)),
               nprob);
  if (aligned) RHQR_CUDA_TRY(launch_pdl(left_refresh_vec_kernel<T>, g, dim3(256), 0, st, ca));
  else RHQR_CUDA_TRY(launch_pdl(left_refresh_kernel<T>, g, dim3(256), 0, st, ca));
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

// SRHT: block j1 owns rows [j1 N2, (j1+1) N2); refresh (or read the refreshed
// column), signs, FWHT, keep samples
template <class T, bool REFRESHED>
__global__ void left_column_srht_kernel(ColArgs a0, const uint32_t *sign_bits, int32_t N2, const int32_t *i2_list,
                                        int32_t d2, T *Ystage) {
  pdl_wait();
  pdl_release();
  const ColArgs a = batch_args<T>(a0);
  Ystage += (int64_t)blockIdx.y * a0.bt.stage;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *v = reinterpret_cast<T *>(smem_raw);
  __shared__ double c_s[1024];
  for (int l = threadIdx.x; l < a.j - a.lo; l += blockDim.x) c_s[l] = a.c[l];
  const T inv_g = (a.j - 1 >= a.lo) ? (T)(1.0 / a.gamma[a.j - 1]) : T(1);
  __syncthreads();
  const int64_t row0 = (int64_t)blockIdx.x * N2;
  for (int t = threadIdx.x; t < N2; t += blockDim.x) {
    int64_t i = row0 + t;
    T val = T(0);
    if (i < a.n) {
      if (REFRESHED) {
        if (i >= a.skm) {
          const T w = ((const T *)a.U)[(int64_t)a.j * a.ldu + i];
          val = ((sign_bits[i >> 5] >> (i & 31)) & 1u) ? -w : w;
        }
      } else {
        T w = refresh_row<T>(a, i, c_s, inv_g);
        if (i < a.m) a.y[i] = (double)w;
        if (i >= a.skm) val = ((sign_bits[i >> 5] >> (i & 31)) & 1u) ? -w : w;
      }
    }
    v[t] = val;
  }
  __syncthreads();
  for (int h = 1; h < N2; h <<= 1) {
    for (int t = threadIdx.x; t < (N2 >> 1); t += blockDim.x) {
      int i = (t / h) * (2 * h) + (t % h);
      T x0 = v[i], x1 = v[i + h];
      v[i] = x0 + x1;
      v[i + h] = x0 - x1;
    }
    __syncthreads();
  }
  T *ys = Ystage + (int64_t)blockIdx.x * d2;
  for (int s = threadIdx.x; s < d2; s += blockDim.x) ys[s] = v[i2_list[s]];
}

// The refreshed column j (stored in U) of problem blockIdx.y: rows >= skm
// signed, segment blockIdx.x transformed by fwht_segment (N2 = 2^LOGN2 >=
// 512), the sampled in-segment positions kept.
template <class T, int LOGN2>
__global__ void __launch_bounds__(1 << (LOGN2 - 4)) column_srht_fwht_kernel(ColArgs a0, const uint32_t *sign_bits,
                                                                            const int32_t *i2_list, int32_t d2,
                                                                            T *Ystage) {
  pdl_wait();
  pdl_release();
  constexpr int N2 = 1 << LOGN2, NT = N2 / 16;
  const ColArgs a = batch_args<T>(a0);
  Ystage += (int64_t)blockIdx.y * a0.bt.stage;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *buf = reinterpret_cast<T *>(smem_raw);
  const int t = threadIdx.x;
  const int64_t row0 = (int64_t)blockIdx.x * N2;
  const T *u = (const T *)a.U + (int64_t)a.j * a.ldu;
  T v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int64_t i = row0 + r * NT + t;
    T val = T(0);
    if (i >= a.skm && i < a.n) {
      val = u[i];
      if ((sign_bits[i >> 5] >> (i & 31)) & 1u) val = -val;
    }
    v[r] = val;
  }
  fwht_segment<T, LOGN2>(v, buf);
  T *ys = Ystage + (int64_t)blockIdx.x * d2;
  for (int s = t; s < d2; s += NT) ys[s] = buf[i2_list[s]];
}

template <class T, int LOGN2>
static rhqr_status launch_column_fwht(const ColArgs &ca, const SketchView &v, T *stage, unsigned nprob,
                                      cudaStream_t st) {
  const size_t smem = sizeof(T) << LOGN2;
  if (smem > 48 * 1024)
    RHQR_CUDA_TRY(cudaFuncSetAttribute(column_srht_fwht_kernel<T, LOGN2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
  RHQR_CUDA_TRY(launch_pdl(column_srht_fwht_kernel<T, LOGN2>, dim3((unsigned)v.N1, nprob), dim3(1 << (LOGN2 - 4)),
                           smem, st, ca, v.sign_bits, v.i2_list, v.d2, stage));
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

// Stage A of the SRHT of the refreshed column(s) (nprob problems of a batch):
// the register / shuffle transform for segments of 512 entries or more, else
// the shared-memory kernel.
template <class T>
static rhqr_status column_srht(const ColArgs &ca, const SketchView &v, T *stage, unsigned nprob, cudaStream_t st) {
  switch (v.N2) {
    case 8192: return launch_column_fwht<T, 13>(ca, v, stage, nprob, st);
    case 4096: return launch_column_fwht<T, 12>(ca, v, stage, nprob, st);
    case 2048: return launch_column_fwht<T, 11>(ca, v, stage, nprob, st);
    case 1024: return launch_column_fwht<T, 10>(ca, v, stage, nprob, st);
    case 512: return launch_column_fwht<T, 9>(ca, v, stage, nprob, st);
    default: break;
  }
  const size_t smem = (size_t)v.N2 * sizeof(T);
  RHQR_CUDA_TRY(launch_pdl(left_column_srht_kernel<T, true>, dim3((unsigned)v.N1, nprob), dim3(512), smem, st, ca,
                           v.sign_bits, v.N2, v.i2_list, v.d2, stage));
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

// Stage B of the SRHT of one column per problem (blockIdx.y): sampled row r
// = i1 N2 + i2 sums its N1 segment values with the signs (-1)^popc(i1 & j1).
// One warp per sampled row: lane l adds j1 = l, l + 32, ... and the lane sums
// meet in a fixed tree.
template <class T>
__global__ void left_srht_combine_kernel(const T *Ystage, int32_t N1, int32_t d2, const int32_t *sample_i1,
                                         const int32_t *sample_slot, int32_t k, int32_t m, double scale, double *y,
                                         int64_t bs_stage = 0, int64_t bs_y = 0) {
  pdl_wait();
  pdl_release();
  Ystage += (int64_t)blockIdx.y * bs_stage;
  y += (int64_t)blockIdx.y * bs_y;
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= k) return;
  const int i1 = sample_i1[r], slot = sample_slot[r];
  double acc = 0.0;
  for (int j1 = lane; j1 < N1; j1 += 32) {
    const double t = (double)Ystage[(int64_t)j1 * d2 + slot];
    acc += (__popc(i1 & j1) & 1) ? -t : t;
  }
  acc = warp_sum(acc);
  if (lane == 0) y[m + r] = acc * scale;
}

// Gaussian: block owns rows [b*RB, (b+1)*RB); partial[b][r] = sum_i G[r, i] w_i over rows i >= m
constexpr int LG_RB = 256;
template <class T, class TG>
__global__ void __launch_bounds__(LG_RB) left_column_gauss_kernel(ColArgs a0, const TG *G, int64_t ldg, int32_t k,
                                                                  double *part) {
  pdl_wait();
  const ColArgs a = batch_args<T>(a0);
  part += (int64_t)blockIdx.y * a0.bt.stage;
  __shared__ double w_s[LG_RB];
  __shared__ double c_s[1024];
  for (int l = threadIdx.x; l < a.j - a.lo; l += blockDim.x) c_s[l] = a.c[l];
  const T inv_g = (a.j - 1 >= a.lo) ? (T)(1.0 / a.gamma[a.j - 1]) : T(1);
  __syncthreads();
  const int64_t row0 = (int64_t)blockIdx.x * LG_RB;
  int64_t i = row0 + threadIdx.x;
  double wd = 0.0;
  if (i < a.n) {
    T w = refresh_row<T>(a, i, c_s, inv_g);
    if (i < a.m) a.y[i] = (double)w;
    if (i >= a.skm) wd = (double)w;
  }
  w_s[threadIdx.x] = wd;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = LG_RB / 32;
  const int64_t rows = min((int64_t)LG_RB, a.n - row0);
  for (int r = wid; r < k; r += nw) {
    double acc = 0.0;
    for (int t = lane; t < rows; t += 32) acc += to_f64<TG>(G[(int64_t)r * ldg + row0 + t]) * w_s[t];
    acc = warp_sum(acc);
    if (lane == 0) part[(int64_t)blockIdx.x * k + r] = acc;
  }
}

static __global__ void left_gauss_reduce_kernel(const double *part, int32_t nb, int32_t k, int32_t m, double scale,
                                                double *y, int64_t bs_stage = 0, int64_t bs_y = 0) {
  pdl_wait();
  pdl_release();
  part += (int64_t)blockIdx.y * bs_stage;
  y += (int64_t)blockIdx.y * bs_y;
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= k) return;
  double acc = 0.0;
  for (int b = 0; b < nb; ++b) acc += part[(int64_t)b * k + r];
  y[m + r] = acc * scale;
}

// final deferred scale of column j: u = u~ / gamma (rows >= j+1), u_j = 1 (or gamma/div)
template <class T>
__global__ void left_scale_last_kernel(T *U, int64_t ldu, int64_t n, int32_t j, const double *gamma, int32_t unit,
                                       int64_t bs_U = 0, int64_t bs_vec = 0) {
  pdl_wait();
  U += (int64_t)blockIdx.y * bs_U;
  gamma += (int64_t)blockIdx.y * bs_vec;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T *up = U + (int64_t)j * ldu + i;
  T inv_g = (T)(1.0 / gamma[j]);
  *up = (i < j) ? T(0) : ((i == j && unit) ? T(1) : *up * inv_g);
}

}  // namespace rhqr
