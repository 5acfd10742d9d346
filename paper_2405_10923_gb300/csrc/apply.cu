// High-dimensional row passes of RHQR.
//
//   solve : Y = X Tri^{-1} for upper-triangular Tri (m x m).  With Tri = R this
//           forms Q = W R^{-1} (recRHQR's Q, Section 3.3); with Tri = M =
//           ut(T^t S^t Z) it is the column recursion of Algorithm 6 that gives
//           U_2 from W_2 = U_2 M.  Each row is an independent forward
//           substitution, i.e. backward stable row by row.
//   solve+mul : the same, then Q_2 = -U_2 G with G = T U_1^t (Section 3.2).
//   mul   : Q = [I_m; 0] - U G (thin Q of left-looking RHQR, Section 3.2).
//
// One thread owns one row.  The row lives in shared memory (column-major in
// the block: xs[j * RB + t]); columns are processed in panels of 32 so that
// the off-diagonal update has 32 independent accumulators per thread.  The
// small matrices are read transposed (row l contiguous) and padded to a
// multiple of 32 with an identity, so panels need no bounds checks.
#include "apply.cuh"
#include "solve_inv_tc.cuh"
#include "common.cuh"

namespace rhqr {

constexpr int PB = 32;  // panel width

template <class T>
__device__ __forceinline__ void load_panel(const T *p, T (&r)[PB]);
template <>
__device__ __forceinline__ void load_panel<float>(const float *p, float (&r)[PB]) {
  const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
  for (int i = 0; i < PB / 4; ++i) {
    float4 v = __ldg(q + i);
    r[4 * i] = v.x;
    r[4 * i + 1] = v.y;
    r[4 * i + 2] = v.z;
    r[4 * i + 3] = v.w;
  }
}
template <>
__device__ __forceinline__ void load_panel<double>(const double *p, double (&r)[PB]) {
  const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
  for (int i = 0; i < PB / 2; ++i) {
    double2 v = __ldg(q + i);
    r[2 * i] = v.x;
    r[2 * i + 1] = v.y;
  }
}

// MODE 0: out1 = X Tri^{-1}
// MODE 1: Y = X Tri^{-1}; out1 = Y (if non-null); out2 = -Y G
// MODE 2: out2 = E - X G, E_ij = 1 if global row i == j (i < m)
template <class T, int MODE>
__global__ void __launch_bounds__(128) row_pass_kernel(const T *X, int64_t ldx, int64_t row_begin, int64_t nrows,
                                                       int32_t m, int32_t mp, const T *TriT, const T *GT,
                                                       T *out1, int64_t ld1, T *out2, int64_t ld2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  const int RB = blockDim.x, t = threadIdx.x;
  const int64_t i = row_begin + (int64_t)blockIdx.x * RB + t;
  const bool live = (i < row_begin + nrows);
  for (int j = 0; j < mp; ++j) xs[j * RB + t] = (live && j < m) ? X[(int64_t)j * ldx + i] : T(0);

  if (MODE == 0 || MODE == 1) {
    for (int J0 = 0; J0 < mp; J0 += PB) {
      T acc[PB];
#pragma unroll
      for (int jj = 0; jj < PB; ++jj) acc[jj] = xs[(J0 + jj) * RB + t];
      for (int l = 0; l < J0; ++l) {
        T r[PB];
        load_panel<T>(TriT + (int64_t)l * mp + J0, r);
        T yl = xs[l * RB + t];
#pragma unroll
        for (int jj = 0; jj < PB; ++jj) acc[jj] -= yl * r[jj];
      }
#pragma unroll
      for (int jj = 0; jj < PB; ++jj) {
        T r[PB];
        load_panel<T>(TriT + (int64_t)(J0 + jj) * mp + J0, r);  // row J0+jj of Tri, panel J0
        acc[jj] = acc[jj] / r[jj];
#pragma unroll
        for (int q = jj + 1; q < PB; ++q) acc[q] -= acc[jj] * r[q];
      }
#pragma unroll
      for (int jj = 0; jj < PB; ++jj) xs[(J0 + jj) * RB + t] = acc[jj];
    }
    if (MODE == 0 || out1 != nullptr) {
      if (live)
        for (int j = 0; j < m; ++j) out1[(int64_t)j * ld1 + i] = xs[j * RB + t];
    }
  }
  if (MODE == 1 || MODE == 2) {
    const T sign = (MODE == 1) ? T(-1) : T(1);
    for (int J0 = 0; J0 < mp; J0 += PB) {
      T acc[PB];
#pragma unroll
      for (int jj = 0; jj < PB; ++jj) acc[jj] = T(0);
      for (int l = 0; l < J0 + PB; ++l) {
        T r[PB];
        load_panel<T>(GT + (int64_t)l * mp + J0, r);
        T yl = xs[l * RB + t];
#pragma unroll
        for (int jj = 0; jj < PB; ++jj) acc[jj] += yl * r[jj];
      }
      if (live) {
#pragma unroll
        for (int jj = 0; jj < PB; ++jj) {
          int j = J0 + jj;
          if (j < m) {
            T v = (MODE == 1) ? sign * acc[jj] : (((int64_t)j == i) ? T(1) : T(0)) - acc[jj];
            out2[(int64_t)j * ld2 + i] = v;
          }
        }
      }
    }
  }
}

// Padded transpose of an m x m float64 matrix (ld = m) into T (mp x mp,
// row-major): out[l * mp + j] = A[l, j] for l, j < m; identity on the padding.
// `upper` zeroes the strictly lower part.
template <class T>
__global__ void pad_transpose_kernel(const double *A, int32_t m, int32_t mp, int upper, T *out) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)mp * mp) return;
  int l = (int)(idx / mp), j = (int)(idx % mp);
  double v;
  if (l < m && j < m) v = (upper && l > j) ? 0.0 : A[(int64_t)j * m + l];
  else v = (l == j) ? 1.0 : 0.0;
  out[idx] = (T)v;
}

// U[i, j] = S[i, j] for i < m (cast to T)
template <class T>
__global__ void top_from_s_kernel(const double *S, int64_t lds, int32_t m, T *U, int64_t ldu) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * m) return;
  int j = (int)(idx / m), i = (int)(idx % m);
  U[(int64_t)j * ldu + i] = (T)S[(int64_t)j * lds + i];
}

// ---------------------------------------------------------------------------

int32_t padded_m(int32_t m) { return (int32_t)ceil_div(m, PB) * PB; }

size_t small_padded_bytes(int32_t m) { return (size_t)padded_m(m) * padded_m(m) * sizeof(double); }

template <class T>
static int rows_per_block(int32_t mp) {
  size_t per_row = (size_t)mp * sizeof(T);
  int rb = 128;
  while (rb > 32 && per_row * rb > 96 * 1024) rb >>= 1;
  return rb;
}

template <class T>
rhqr_status pad_transpose_to(const double *A, int32_t m, int32_t mp, int upper, T *out, cudaStream_t st) {
  if (mp < m) return RHQR_EINVAL;
  pad_transpose_kernel<T><<<(unsigned)ceil_div((int64_t)mp * mp, 256), 256, 0, st>>>(A, m, mp, upper, out);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}
template <class T>
rhqr_status pad_transpose(const double *A, int32_t m, int upper, T *out, cudaStream_t st) {
  return pad_transpose_to<T>(A, m, padded_m(m), upper, out, st);
}
template rhqr_status pad_transpose<float>(const double *, int32_t, int, float *, cudaStream_t);
template rhqr_status pad_transpose<double>(const double *, int32_t, int, double *, cudaStream_t);
template rhqr_status pad_transpose_to<float>(const double *, int32_t, int32_t, int, float *, cudaStream_t);
template rhqr_status pad_transpose_to<double>(const double *, int32_t, int32_t, int, double *, cudaStream_t);

template <class T, int MODE>
static rhqr_status launch_rows(const T *X, int64_t ldx, int64_t row_begin, int64_t nrows, int32_t m, const T *TriT,
                               const T *GT, T *out1, int64_t ld1, T *out2, int64_t ld2, cudaStream_t st) {
  if (nrows <= 0) return RHQR_OK;
  int32_t mp = padded_m(m);
  int rb = rows_per_block<T>(mp);
  size_t smem = (size_t)mp * rb * sizeof(T);
  if (smem > 200 * 1024) return RHQR_ENOTSUP;
  RHQR_CUDA_TRY(cudaFuncSetAttribute(row_pass_kernel<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  unsigned grid = (unsigned)ceil_div(nrows, rb);
  row_pass_kernel<T, MODE><<<grid, rb, smem, st>>>(X, ldx, row_begin, nrows, m, mp, TriT, GT, out1, ld1, out2, ld2);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

template <class T>
rhqr_status rows_solve(const T *X, int64_t ldx, int64_t row_begin, int64_t nrows, int32_t m, const T *TriT, T *Y,
                       int64_t ldy, cudaStream_t st) {
  return launch_rows<T, 0>(X, ldx, row_begin, nrows, m, TriT, nullptr, Y, ldy, nullptr, 0, st);
}
template <class T>
rhqr_status rows_solve_mul(const T *X, int64_t ldx, int64_t row_begin, int64_t nrows, int32_t m, const T *TriT,
                           const T *GT, T *U, int64_t ldu, T *Q, int64_t ldq, cudaStream_t st) {
  return launch_rows<T, 1>(X, ldx, row_begin, nrows, m, TriT, GT, U, ldu, Q, ldq, st);
}
template <class T>
rhqr_status rows_form_q(const T *U, int64_t ldu, int64_t row_begin, int64_t nrows, int32_t m, const T *GT, T *Q,
                        int64_t ldq, cudaStream_t st) {
  return launch_rows<T, 2>(U, ldu, row_begin, nrows, m, nullptr, GT, nullptr, 0, Q, ldq, st);
}
template <class T>
rhqr_status top_from_s(const double *S, int64_t lds, int32_t m, T *U, int64_t ldu, cudaStream_t st) {
  top_from_s_kernel<T><<<(unsigned)ceil_div((int64_t)m * m, 256), 256, 0, st>>>(S, lds, m, U, ldu);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

// Q = [I_m; 0] - U G for an upper-triangular G (m x m float64, ld m; G is
// overwritten).  float32 with m <= 256: on the tensor cores as the product
// with -G (rows_solve_inv_tc, the explicit-inverse solve, whose operand is an
// upper-triangular matrix with a nonzero diagonal: here diag(G)_j = t_jj
// u_jj != 0), then the identity block added; otherwise the SIMT row pass.
static __global__ void negate_kernel(double *A, int64_t count) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) A[e] = -A[e];
}
template <class T>
static __global__ void add_identity_kernel(T *Q, int64_t ldq, int32_t m) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) Q[(int64_t)j * ldq + j] += T(1);
}

template <class T>
rhqr_status form_q_from_g(const T *U, int64_t ldu, int64_t n, int32_t m, double *Gm, void *GT, T *Q, int64_t ldq,
                          rhqr_info *info, cudaStream_t st) {
  if (sizeof(T) == 4 && solve_inv_tc_supported(m) && (const void *)U != (const void *)Q) {
    negate_kernel<<<(unsigned)ceil_div((int64_t)m * m, 256), 256, 0, st>>>(Gm, (int64_t)m * m);
    RHQR_LAUNCH_CHECK();
    RHQR_TRY(rows_solve_inv_tc((const float *)U, ldu, n, m, Gm, 0, (float *)Q, ldq, info, kDefaultWaitBudget, st));
    add_identity_kernel<T><<<(unsigned)ceil_div(m, 256), 256, 0, st>>>(Q, ldq, m);
    RHQR_LAUNCH_CHECK();
    return RHQR_OK;
  }
  RHQR_TRY(pad_transpose<T>(Gm, m, 1, (T *)GT, st));
  return rows_form_q<T>(U, ldu, 0, n, m, (const T *)GT, Q, ldq, st);
}

#define RHQR_INST(T)                                                                                          \
  template rhqr_status rows_solve<T>(const T *, int64_t, int64_t, int64_t, int32_t, const T *, T *, int64_t,  \
                                     cudaStream_t);                                                           \
  template rhqr_status rows_solve_mul<T>(const T *, int64_t, int64_t, int64_t, int32_t, const T *, const T *, \
                                         T *, int64_t, T *, int64_t, cudaStream_t);                           \
  template rhqr_status rows_form_q<T>(const T *, int64_t, int64_t, int64_t, int32_t, const T *, T *, int64_t, \
                                      cudaStream_t);                                                          \
  template rhqr_status top_from_s<T>(const double *, int64_t, int32_t, T *, int64_t, cudaStream_t);          \
  template rhqr_status form_q_from_g<T>(const T *, int64_t, int64_t, int32_t, double *, void *, T *, int64_t,   \
                                        rhqr_info *, cudaStream_t);
RHQR_INST(float)
RHQR_INST(double)
#undef RHQR_INST

}  // namespace rhqr
