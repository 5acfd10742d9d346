// Matrix-free 2-D convection-diffusion operator of the RHQR-GMRES workload
// (5-point central differences on a g x g interior grid, zero Dirichlet
// boundary, scaled by h^2) and the restart residual R = B - A X with its
// norms.  Memory-bound: one thread per grid point and right-hand side, the
// four neighbours read through the read-only cache (rows r +- 1 share cache
// lines with r, rows r +- g with the neighbouring warps' loads).
#include <algorithm>

#include "common.cuh"

namespace rhqr {

template <class T>
__device__ __forceinline__ double stencil_at(const T *x, int32_t g, double c, int64_t r) {
  const int64_t iy = r / g, ix = r - iy * g;
  double acc = 4.0 * (double)__ldg(x + r);
  if (ix > 0) acc -= (1.0 + c) * (double)__ldg(x + r - 1);
  if (ix + 1 < g) acc -= (1.0 - c) * (double)__ldg(x + r + 1);
  if (iy > 0) acc -= (1.0 + c) * (double)__ldg(x + r - g);
  if (iy + 1 < g) acc -= (1.0 - c) * (double)__ldg(x + r + g);
  return acc;
}

template <class T>
__global__ void __launch_bounds__(256) stencil_kernel(int32_t g, double c, const T *X, T *Y) {
  const int64_t n = (int64_t)g * g;
  const int64_t b = blockIdx.y;
  const T *x = X + b * n;
  T *y = Y + b * n;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
    y[r] = (T)stencil_at(x, g, c, r);
}

// R = B - A X (formed in float64, stored in R's type TR); partial[(b * nblk +
// block) * 2 + {0, 1}] = this block's sums of r^2 and b^2 of the float64
// values (fixed order: grid-stride loop, then the block tree)
template <class T, class TR>
__global__ void __launch_bounds__(256) stencil_residual_kernel(int32_t g, double c, const T *B, const T *X, TR *R,
                                                               double *partial) {
  __shared__ double red[32];
  const int64_t n = (int64_t)g * g;
  const int64_t b = blockIdx.y;
  const T *x = X + b * n;
  const T *bb = B + b * n;
  TR *rr = R + b * n;
  double sr = 0.0, sb = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const double bv = (double)bb[r];
    const double rv = bv - stencil_at(x, g, c, r);
    rr[r] = (TR)rv;
    sr += rv * rv;
    sb += bv * bv;
  }
  sr = block_sum(sr, red);
  sb = block_sum(sb, red);
  if (threadIdx.x == 0) {
    partial[(b * gridDim.x + blockIdx.x) * 2] = sr;
    partial[(b * gridDim.x + blockIdx.x) * 2 + 1] = sb;
  }
}

__global__ void stencil_norms_kernel(const double *partial, int32_t nblk, double *norms) {
  const int64_t b = blockIdx.x;
  if (threadIdx.x >= 2) return;
  double acc = 0.0;
  for (int i = 0; i < nblk; ++i) acc += partial[(b * nblk + i) * 2 + threadIdx.x];
  norms[b * 2 + threadIdx.x] = sqrt(acc);
}

static int32_t residual_blocks(int32_t g) {
  return (int32_t)std::min<int64_t>(ceil_div((int64_t)g * g, 256), 152 * 4);
}

}  // namespace rhqr

using namespace rhqr;

extern "C" rhqr_status rhqr_stencil_apply(int32_t g, double pe, const void *X, int32_t dt, int32_t nrhs, void *Y,
                                          rhqr_stream_t stream) {
  if (g < 1 || nrhs < 1 || nrhs > 65535 || X == nullptr || Y == nullptr || (dt != RHQR_F64 && dt != RHQR_F32))
    return RHQR_EINVAL;
  const double c = pe / (2.0 * (g + 1));
  const dim3 grid((unsigned)std::min<int64_t>(ceil_div((int64_t)g * g, 256), 152 * 8), (unsigned)nrhs);
  cudaStream_t st = (cudaStream_t)stream;
  if (dt == RHQR_F64)
    stencil_kernel<double><<<grid, 256, 0, st>>>(g, c, (const double *)X, (double *)Y);
  else
    stencil_kernel<float><<<grid, 256, 0, st>>>(g, c, (const float *)X, (float *)Y);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

extern "C" rhqr_status rhqr_stencil_residual_workspace(int32_t g, int32_t nrhs, size_t *bytes) {
  if (g < 1 || nrhs < 1 || bytes == nullptr) return RHQR_EINVAL;
  *bytes = sizeof(double) * 2 * (size_t)residual_blocks(g) * (size_t)nrhs;
  return RHQR_OK;
}

extern "C" rhqr_status rhqr_stencil_residual(int32_t g, double pe, const void *B, const void *X, int32_t dt,
                                             int32_t nrhs, void *R, int32_t rdt, double *norms, void *work,
                                             size_t work_bytes, rhqr_stream_t stream) {
  if (g < 1 || nrhs < 1 || nrhs > 65535 || B == nullptr || X == nullptr || R == nullptr || norms == nullptr ||
      (dt != RHQR_F64 && dt != RHQR_F32) || (rdt != RHQR_F64 && rdt != RHQR_F32))
    return RHQR_EINVAL;
  const int32_t nblk = residual_blocks(g);
  if (work == nullptr || work_bytes < sizeof(double) * 2 * (size_t)nblk * (size_t)nrhs) return RHQR_ENOMEM;
  const double c = pe / (2.0 * (g + 1));
  cudaStream_t st = (cudaStream_t)stream;
  const dim3 grid((unsigned)nblk, (unsigned)nrhs);
  double *part = (double *)work;
  if (dt == RHQR_F64 && rdt == RHQR_F64)
    stencil_residual_kernel<double, double><<<grid, 256, 0, st>>>(g, c, (const double *)B, (const double *)X,
                                                                  (double *)R, part);
  else if (dt == RHQR_F64)
    stencil_residual_kernel<double, float><<<grid, 256, 0, st>>>(g, c, (const double *)B, (const double *)X,
                                                                 (float *)R, part);
  else if (rdt == RHQR_F64)
    stencil_residual_kernel<float, double><<<grid, 256, 0, st>>>(g, c, (const float *)B, (const float *)X,
                                                                 (double *)R, part);
  else
    stencil_residual_kernel<float, float><<<grid, 256, 0, st>>>(g, c, (const float *)B, (const float *)X,
                                                                (float *)R, part);
  RHQR_LAUNCH_CHECK();
  stencil_norms_kernel<<<(unsigned)nrhs, 32, 0, st>>>(part, nblk, norms);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}
