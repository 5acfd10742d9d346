// BLAS2-RGS (Algorithm 9, Section 6): the RHQR of [0_m; W] written on W, which
// reproduces randomized Gram-Schmidt in exact arithmetic and keeps in T the
// loss of sketched orthogonality.  Column j:
//   z = Omega w_j,  r = T_{0:j,0:j}^t S_{0:j}^t z,  w = w_j - Q_{0:j} r,
//   z = Omega w,  rho = ||z||,  q_j = w / rho,  s_j = z / rho,
//   R_{0:j,j} = r,  R_jj = rho,  T_{0:j,j} = -T_{0:j,0:j} S_{0:j}^t s_j,  T_jj = 1
// with Omega = Omega_full of the sketch handle (no exact top block).  The
// sketches are the library's SIMT sketch of one column; the small products,
// the update of the column and the normalisation are one-block kernels and one
// row-parallel kernel per column.
#include "common.cuh"
#include "sketch.cuh"

namespace rhqr {

const SketchView *sketch_view_of(rhqr_sketch s);

namespace rgs {

// r = T_{0:j,0:j}^t (S_{0:j}^t z): v_i = s_i . z, r_l = sum_{i <= l} T_il v_i
__global__ void coef_kernel(const double *T, int32_t m, const double *S, int32_t k, int32_t j, const double *z,
                            double *v, double *r) {
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    double acc = 0.0;
    for (int e = 0; e < k; ++e) acc += S[(int64_t)i * k + e] * z[e];
    v[i] = acc;
  }
  __syncthreads();
  for (int l = threadIdx.x; l < j; l += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i <= l; ++i) acc += T[(int64_t)l * m + i] * v[i];
    r[l] = acc;
  }
}

// w = w_j - Q_{0:j} r
template <class Tw>
__global__ void update_kernel(const Tw *wj, const Tw *Q, int64_t ldq, int64_t n, int32_t j, const double *r, Tw *w) {
  __shared__ double rs[1024];
  for (int l = threadIdx.x; l < j; l += blockDim.x) rs[l] = r[l];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = (double)wj[i];
  for (int l = 0; l < j; ++l) acc -= (double)Q[(int64_t)l * ldq + i] * rs[l];
  w[i] = (Tw)acc;
}

// rho = ||z|| (fixed-order block reduction), s_j = z / rho, column j of R and T
__global__ void finish_kernel(const double *z, int32_t k, int32_t j, int32_t m, const double *r, double *S,
                              double *R, double *T, double *rho_out, double *v, rhqr_info *info) {
  __shared__ double red[256];
  __shared__ double rho_s;
  double acc = 0.0;
  for (int e = threadIdx.x; e < k; e += blockDim.x) acc += z[e] * z[e];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double rho = sqrt(red[0]);
    rho_s = rho;
    *rho_out = rho;
    if (rho == 0.0 || !isfinite(rho)) set_status(info, rho == 0.0 ? RHQR_EBREAKDOWN : RHQR_ENONFINITE, j);
  }
  __syncthreads();
  const double rho = rho_s;
  for (int e = threadIdx.x; e < k; e += blockDim.x) S[(int64_t)j * k + e] = z[e] / rho;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    R[(int64_t)j * m + i] = i < j ? r[i] : (i == j ? rho : 0.0);
  }
  __syncthreads();
  // v_i = s_i . s_j (i < j), then T_{0:j,j} = -T_{0:j,0:j} v, T_jj = 1
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    double a = 0.0;
    for (int e = 0; e < k; ++e) a += S[(int64_t)i * k + e] * S[(int64_t)j * k + e];
    v[i] = a;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double t = 0.0;
    if (i < j)
      for (int l = i; l < j; ++l) t += T[(int64_t)l * m + i] * v[l];
    T[(int64_t)j * m + i] = i < j ? -t : (i == j ? 1.0 : 0.0);
  }
}

template <class Tw>
__global__ void scale_kernel(const Tw *w, int64_t n, const double *rho, Tw *q) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] = (Tw)((double)w[i] / *rho);
}

}  // namespace rgs

static size_t rgs_workspace(const SketchView &v, int32_t wt, int64_t n, int32_t m) {
  Carver c(nullptr, 0);
  c.take<char>(sketch_apply_workspace_bytes(v, 0, wt, n, 1));
  c.take<double>((size_t)v.k);      // z
  c.take<double>(2 * (size_t)m);    // r, v
  c.take<double>(1);                // rho
  c.take<char>((size_t)n * dtype_size(wt));  // w
  return c.used() + 256;
}

template <class Tw>
static rhqr_status rgs_typed(const SketchView &v, const Tw *W, int64_t n, int32_t m, int64_t ldw, Tw *Q, int64_t ldq,
                             double *R, double *T, double *S, void *ws, size_t ws_bytes, rhqr_info *info,
                             int32_t wt, cudaStream_t st) {
  const size_t skb = sketch_apply_workspace_bytes(v, 0, wt, n, 1);
  Carver c(ws, ws_bytes);
  void *skws = c.take<char>(skb);
  double *z = c.take<double>((size_t)v.k);
  double *r = c.take<double>((size_t)m);
  double *vv = c.take<double>((size_t)m);
  double *rho = c.take<double>(1);
  Tw *w = reinterpret_cast<Tw *>(c.take<char>((size_t)n * sizeof(Tw)));
  if (c.overflow()) return RHQR_ENOMEM;
  const unsigned grid = (unsigned)ceil_div(n, (int64_t)256);
  for (int32_t j = 0; j < m; ++j) {
    const Tw *wj = W + (int64_t)j * ldw;
    if (j > 0) {
      RHQR_TRY(sketch_apply_simt(v, 0, wj, wt, n, 1, n, z, v.k, skws, skb, st));
      rgs::coef_kernel<<<1, 256, 0, st>>>(T, m, S, v.k, j, z, vv, r);
      RHQR_LAUNCH_CHECK();
    }
    rgs::update_kernel<Tw><<<grid, 256, 0, st>>>(wj, Q, ldq, n, j, r, w);
    RHQR_LAUNCH_CHECK();
    RHQR_TRY(sketch_apply_simt(v, 0, w, wt, n, 1, n, z, v.k, skws, skb, st));
    rgs::finish_kernel<<<1, 256, 0, st>>>(z, v.k, j, m, r, S, R, T, rho, vv, info);
    RHQR_LAUNCH_CHECK();
    rgs::scale_kernel<Tw><<<grid, 256, 0, st>>>(w, n, rho, Q + (int64_t)j * ldq);
    RHQR_LAUNCH_CHECK();
  }
  return RHQR_OK;
}

}  // namespace rhqr

using namespace rhqr;

extern "C" {

rhqr_status rhqr_blas2_rgs_workspace(rhqr_sketch s, int32_t wt, int64_t n, int32_t m, size_t *bytes) {
  if (s == nullptr || bytes == nullptr || (wt != RHQR_F64 && wt != RHQR_F32) || m < 1 || n <= m) return RHQR_EINVAL;
  const SketchView &v = *sketch_view_of(s);
  // Omega Q (k x m) can only have orthonormal columns when k >= m
  if (m > 1024 || m > v.k || (v.kind == RHQR_SKETCH_GAUSSIAN && n != v.n) || (v.kind == RHQR_SKETCH_SRHT && n > v.N))
    return RHQR_EINVAL;
  *bytes = rgs_workspace(v, wt, n, m);
  return RHQR_OK;
}

rhqr_status rhqr_blas2_rgs(rhqr_sketch s, const void *W, int32_t wt, int64_t n, int32_t m, int64_t ldw, void *Q,
                           int64_t ldq, double *R, double *T, double *S, void *ws, size_t ws_bytes, rhqr_info *info,
                           rhqr_stream_t stream) {
  size_t need = 0;
  RHQR_TRY(rhqr_blas2_rgs_workspace(s, wt, n, m, &need));
  if (W == nullptr || Q == nullptr || R == nullptr || T == nullptr || S == nullptr || info == nullptr)
    return RHQR_EINVAL;
  if (ldw < n || ldq < n) return RHQR_EINVAL;
  if (ws == nullptr || ws_bytes < need) return RHQR_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  RHQR_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(rhqr_info), st));
  const SketchView &v = *sketch_view_of(s);
  if (wt == RHQR_F64)
    return rgs_typed<double>(v, (const double *)W, n, m, ldw, (double *)Q, ldq, R, T, S, ws, ws_bytes, info, wt, st);
  return rgs_typed<float>(v, (const float *)W, n, m, ldw, (float *)Q, ldq, R, T, S, ws, ws_bytes, info, wt, st);
}

}  // extern "C"
