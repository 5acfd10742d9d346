// Small FP64 side of recRHQR (Algorithm 6) on the GPU.
//
// hqr_coop_kernel: Householder QR of Z ((k+m) x m) with the conventions of
//   Algorithm 2 applied to Psi = I: column j gets sigma = sign(z_jj) (sign(0) =
//   +1), rho = ||z_{j:}||, gamma = z_jj + sigma rho, v = (z_{j:})/gamma with
//   v_j = 1 (or the ||v|| = sqrt 2 scaling), beta = 1 + |z_jj|/rho,
//   r_jj = -sigma rho; the trailing columns get (I - beta v v^t).  Rows are
//   spread over the blocks of one cooperative launch; every column costs two
//   bounded grid barriers.  The partial sums are combined in a fixed order,
//   so the result does not depend on timing.
// T factor: Prop. "generalcompactwoodburry" gives (Psi U)^t Psi U = T^{-1} + T^{-t},
//   i.e. T^{-1} = sut(S^t S) + diag(1/beta); T is obtained column by column by
//   back substitution (columns are independent).
// householder_qr_small uses the blocked version (hqr_blocked.cu) where its
//   cluster fits.
// Products of small triangular matrices (R accumulation over passes,
//   G = T U_1^t, M = ut(T^t S^t Z)) and float32 copies for the row solves.
#include "common.cuh"
#include "small.cuh"

namespace rhqr {

struct HqrArgs {
  double *A;  // p x m working copy, ld = p (overwritten)
  int64_t p;
  int32_t m;
  double *S;  // p x m Householder vectors, ld = lds
  int64_t lds;
  double *R;     // m x m
  double *beta;  // m
  double *part;  // gridDim.x * (m + 1)
  unsigned int *bar;
  int *abort_flag;
  rhqr_info *info;
  long long budget;
  int32_t scaling;
};

__global__ void __launch_bounds__(256) hqr_coop_kernel(HqrArgs a) {
  __shared__ double red[32];
  __shared__ double vloc_scale[2];
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int64_t p = a.p;
  const int m = a.m;
  const int64_t per = (p + G - 1) / G;
  const int64_t r0 = min(p, (int64_t)b * per), r1 = min(p, r0 + per);
  double *A = a.A;
  for (int j = 0; j < m; ++j) {
    // ---- phase 1: partial ||z_{j:}||^2 over this block's rows
    double s = 0.0;
    for (int64_t i = max(r0, (int64_t)j) + tid; i < r1; i += nt) {
      double v = A[(int64_t)j * p + i];
      s += v * v;
    }
    s = block_sum(s, red);
    if (tid == 0) a.part[(int64_t)b * (m + 1) + m] = s;
    if (!grid_barrier(a.bar, a.budget, a.info, a.abort_flag)) return;
    // ---- phase 2: every block forms rho, sigma, gamma, beta identically
    if (tid == 0) {
      double ss = 0.0;
      for (int bb = 0; bb < G; ++bb) ss += a.part[(int64_t)bb * (m + 1) + m];
      vloc_scale[0] = ss;
    }
    __syncthreads();
    const double rho = sqrt(vloc_scale[0]);
    const double zjj = A[(int64_t)j * p + j];
    if (!isfinite(rho) || !isfinite(zjj)) {
      if (b == 0 && tid == 0) set_status(a.info, RHQR_ENONFINITE, j);
      return;
    }
    if (rho == 0.0) {
      if (b == 0 && tid == 0) set_status(a.info, RHQR_EBREAKDOWN, j);
      return;
    }
    const double sigma = zjj < 0.0 ? -1.0 : 1.0;
    const double gamma = zjj + sigma * rho;
    const double div = (a.scaling == 0) ? gamma : sqrt(rho * (rho + fabs(zjj)));
    const double beta = (a.scaling == 0) ? 1.0 + fabs(zjj) / rho : 1.0;
    if (b == 0 && tid == 0) a.beta[j] = beta;
    for (int64_t i = r0 + tid; i < r1; i += nt) {
      double *aij = A + (int64_t)j * p + i;
      if (i < j) {
        if (i < m) a.R[(int64_t)j * m + i] = *aij;
        a.S[(int64_t)j * a.lds + i] = 0.0;
      } else {
        double v = (i == j) ? gamma / div : *aij / div;
        *aij = v;
        a.S[(int64_t)j * a.lds + i] = v;
        if (i == j) a.R[(int64_t)j * m + j] = -sigma * rho;
        else if (i < m) a.R[(int64_t)j * m + i] = 0.0;
      }
    }
    __syncthreads();
    // partial dots v . A[:, c] for the trailing columns c > j
    for (int c = j + 1 + tid; c < m; c += nt) {
      double d = 0.0;
      for (int64_t i = max(r0, (int64_t)j); i < r1; ++i) d += A[(int64_t)j * p + i] * A[(int64_t)c * p + i];
      a.part[(int64_t)b * (m + 1) + c] = d;
    }
    if (!grid_barrier(a.bar, a.budget, a.info, a.abort_flag)) return;
    // ---- phase 3: A[:, c] -= beta v (v . A[:, c]) on this block's rows
    for (int c = j + 1 + tid; c < m; c += nt) {
      double w = 0.0;
      for (int bb = 0; bb < G; ++bb) w += a.part[(int64_t)bb * (m + 1) + c];
      w *= beta;
      for (int64_t i = max(r0, (int64_t)j); i < r1; ++i) A[(int64_t)c * p + i] -= A[(int64_t)j * p + i] * w;
    }
    __syncthreads();
  }
}

// SS[i, j] = s_i . s_j for i < j (rows r >= j only: s_j vanishes above j)
__global__ void sts_upper_kernel(const double *S, int64_t lds, int64_t p, int32_t m, double *SS) {
  const int j = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = w; i < j; i += nw) {
    double d = 0.0;
    for (int64_t r = j + lane; r < p; r += 32) d += S[(int64_t)i * lds + r] * S[(int64_t)j * lds + r];
    d = warp_sum(d);
    if (lane == 0) SS[(int64_t)j * m + i] = d;
  }
}

// T column j from T^{-1} = sut(S^t S) + diag(1/beta):
//   T[j, j] = beta_j; T[i, j] = -beta_i sum_{l=i+1..j} SS[i, l] T[l, j], i = j-1..0,
// as a backward column sweep over l (one warp per column).
__global__ void t_from_woodbury_kernel(const double *SS, const double *beta, int32_t m, double *T) {
  // one warp per column, the longest sweeps (largest j) first
  const int jj = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (jj >= m) return;
  const int j = m - 1 - jj;
  column_sweep<4>(SS, m, m, j, beta[j], beta, false, T + (int64_t)j * m);
}

// C = A B for upper-triangular m x m A, B (ld = m); C must not alias A or B.
__global__ void triu_mul_kernel(const double *A, const double *B, int32_t m, double *C) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * m) return;
  int j = (int)(idx / m), i = (int)(idx % m);
  double acc = 0.0;
  for (int l = i; l <= j; ++l) acc += A[(int64_t)l * m + i] * B[(int64_t)j * m + l];
  C[idx] = (i <= j) ? acc : 0.0;
}

// G = T U_1^t with U_1 = S[0:m, 0:m] lower triangular: G[i, j] = sum_{l=i..j} T[i, l] U_1[j, l]
__global__ void t_u1t_kernel(const double *T, const double *S, int64_t lds, int32_t m, double *Gm) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * m) return;
  int j = (int)(idx / m), i = (int)(idx % m);
  double acc = 0.0;
  for (int l = i; l <= j; ++l) acc += T[(int64_t)l * m + i] * S[(int64_t)l * lds + j];
  Gm[idx] = (i <= j) ? acc : 0.0;
}

// StZ[l, j] = sum_{r >= l} S[r, l] Z[r, j]
__global__ void stz_kernel(const double *S, int64_t lds, const double *Z, int64_t ldz, int64_t p, int32_t m,
                           double *StZ) {
  const int j = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int l = w; l < m; l += nw) {
    double d = 0.0;
    for (int64_t r = l + lane; r < p; r += 32) d += S[(int64_t)l * lds + r] * Z[(int64_t)j * ldz + r];
    d = warp_sum(d);
    if (lane == 0) StZ[(int64_t)j * m + l] = d;
  }
}

// M = ut(T^t StZ): M[i, j] = sum_{l <= i} T[l, i] StZ[l, j] for i <= j
__global__ void m_from_stz_kernel(const double *T, const double *StZ, int32_t m, double *M) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * m) return;
  int j = (int)(idx / m), i = (int)(idx % m);
  double acc = 0.0;
  if (i <= j)
    for (int l = 0; l <= i; ++l) acc += T[(int64_t)i * m + l] * StZ[(int64_t)j * m + l];
  M[idx] = acc;
}

__global__ void cast_f32_kernel(const double *A, int64_t n, float *B) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) B[i] = (float)A[i];
}

__global__ void copy_f64_kernel(const double *A, int64_t n, double *B) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) B[i] = A[i];
}

// copy a p x m column-major block with leading dimensions lda -> ldb
__global__ void copy_f64_2d_kernel(const double *A, int64_t lda, int64_t p, int32_t m, double *B, int64_t ldb) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p * m) return;
  int64_t j = idx / p, i = idx - j * p;
  B[j * ldb + i] = A[j * lda + i];
}

__global__ void info_pass_kernel(rhqr_info *info, int32_t passes) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && info != nullptr && info->status == RHQR_OK) info->passes_done = passes;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static int hqr_grid(int64_t p) {
  static int max_coop = -1;
  if (max_coop < 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, hqr_coop_kernel, 256, 0);
    max_coop = std::max(1, sms * std::max(1, per));
  }
  int64_t want = std::max<int64_t>(1, ceil_div(p, 16));  // >= 16 rows per block
  return (int)std::min<int64_t>(std::min<int64_t>(want, 128), max_coop);
}

size_t hqr_workspace_bytes(int64_t p, int32_t m) {
  Carver c(nullptr, 0);
  c.take<double>((size_t)p * m);
  c.take<double>((size_t)128 * (m + 1));
  c.take<unsigned int>(4);
  return std::max(c.used() + 256, hqr_blocked_workspace_bytes(p, m));
}

rhqr_status copy_f64_2d(const double *A, int64_t lda, int64_t p, int32_t m, double *B, int64_t ldb, cudaStream_t st) {
  copy_f64_2d_kernel<<<(unsigned)ceil_div(p * m, 256), 256, 0, st>>>(A, lda, p, m, B, ldb);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

rhqr_status householder_qr_small(const double *Z, int64_t ldz, int64_t p, int32_t m, double *S, int64_t lds,
                                 double *R, double *beta, int32_t scaling, void *ws, size_t ws_bytes,
                                 rhqr_info *info, long long budget, cudaStream_t st) {
  // blocked panels on clusters of CTAs where they fit, else column by column
  const rhqr_status sb = householder_qr_blocked(Z, ldz, p, m, S, lds, R, beta, scaling, ws, ws_bytes, info, st);
  if (sb != RHQR_ENOTSUP) return sb;
  Carver c(ws, ws_bytes);
  double *A = c.take<double>((size_t)p * m);
  double *part = c.take<double>((size_t)128 * (m + 1));
  unsigned int *bar = c.take<unsigned int>(4);
  if (c.overflow()) return RHQR_ENOMEM;
  int64_t tot = p * m;
  copy_f64_2d_kernel<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(Z, ldz, p, m, A, p);
  RHQR_LAUNCH_CHECK();
  RHQR_CUDA_TRY(cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned int), st));
  HqrArgs args{A, p, m, S, lds, R, beta, part, bar, (int *)(bar + 2), info, budget, scaling};
  int grid = hqr_grid(p);
  void *kargs[] = {&args};
  RHQR_CUDA_TRY(cudaLaunchCooperativeKernel((void *)hqr_coop_kernel, dim3(grid), dim3(256), kargs, 0, st));
  count_launch();
  return RHQR_OK;
}

rhqr_status t_factor_small(const double *S, int64_t lds, int64_t p, int32_t m, const double *beta, double *SS,
                           double *T, cudaStream_t st) {
  RHQR_CUDA_TRY(cudaMemsetAsync(SS, 0, sizeof(double) * m * m, st));
  sts_upper_kernel<<<m, 256, 0, st>>>(S, lds, p, m, SS);
  RHQR_LAUNCH_CHECK();
  t_from_woodbury_kernel<<<(unsigned)m, 32, 0, st>>>(SS, beta, m, T);  // spread over the SMs (FP64 issue-bound)
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

rhqr_status triu_mul(const double *A, const double *B, int32_t m, double *C, cudaStream_t st) {
  triu_mul_kernel<<<(unsigned)ceil_div((int64_t)m * m, 256), 256, 0, st>>>(A, B, m, C);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

rhqr_status t_u1t(const double *T, const double *S, int64_t lds, int32_t m, double *Gm, cudaStream_t st) {
  t_u1t_kernel<<<(unsigned)ceil_div((int64_t)m * m, 256), 256, 0, st>>>(T, S, lds, m, Gm);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

rhqr_status m_factor(const double *T, const double *S, int64_t lds, const double *Z, int64_t ldz, int64_t p,
                     int32_t m, double *StZ, double *M, cudaStream_t st) {
  stz_kernel<<<m, 256, 0, st>>>(S, lds, Z, ldz, p, m, StZ);
  RHQR_LAUNCH_CHECK();
  m_from_stz_kernel<<<(unsigned)ceil_div((int64_t)m * m, 256), 256, 0, st>>>(T, StZ, m, M);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

rhqr_status cast_f32(const double *A, int64_t n, float *B, cudaStream_t st) {
  cast_f32_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(A, n, B);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

rhqr_status copy_f64(const double *A, int64_t n, double *B, cudaStream_t st) {
  copy_f64_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(A, n, B);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

// Column equilibration of a sketch: d_j = ||Z[:, j]||_2 (1 for a zero column),
// Z[:, j] /= d_j.  One CTA per column, fixed-order sum.
__global__ void equilibrate_columns_kernel(double *Z, int64_t ldz, int64_t p, double *d) {
  __shared__ double red[32];
  double *z = Z + (int64_t)blockIdx.x * ldz;
  double acc = 0.0;
  for (int64_t r = threadIdx.x; r < p; r += blockDim.x) acc += z[r] * z[r];
  acc = block_sum(acc, red);
  const double nrm = acc > 0.0 ? sqrt(acc) : 1.0;
  for (int64_t r = threadIdx.x; r < p; r += blockDim.x) z[r] = z[r] / nrm;
  if (threadIdx.x == 0) d[blockIdx.x] = nrm;
}

// A[:, j] *= d_j (A rows x m, ld lda)
__global__ void scale_columns_kernel(double *A, int64_t lda, int64_t rows, int32_t m, const double *d) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * m) return;
  const int64_t j = e / rows, i = e - j * rows;
  A[j * lda + i] *= d[j];
}

rhqr_status equilibrate_columns(double *Z, int64_t ldz, int64_t p, int32_t m, double *d, cudaStream_t st) {
  equilibrate_columns_kernel<<<(unsigned)m, 256, 0, st>>>(Z, ldz, p, d);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

rhqr_status scale_columns(double *A, int64_t lda, int64_t rows, int32_t m, const double *d, cudaStream_t st) {
  scale_columns_kernel<<<(unsigned)ceil_div(rows * m, 256), 256, 0, st>>>(A, lda, rows, m, d);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

rhqr_status info_passes(rhqr_info *info, int32_t passes, cudaStream_t st) {
  info_pass_kernel<<<1, 32, 0, st>>>(info, passes);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

}  // namespace rhqr
