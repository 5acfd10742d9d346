// Left-looking trimRHQR (Section 7, the left-looking trimRHQR algorithm) on the
// GPU.
//
// The reflectors are H(u_j, Omega, j) = I - beta_j u_j (Omega u_j)^t
// [0 Omega_{j:n}] (eq. rhousebisbis) with Omega = Omega_full (k x n, no exact
// top block; k may be smaller than m) whose first m columns have unit norm.
// Their left-wise product is I - U Tt^t ut((Omega U)^t Omega) (eq.
// trimrhqrcompactfact), so step j refreshes the input column w_j with
//   v = ut((Omega U_j)^t Omega) w_j,  v_i = s_i . (Omega w_j) - sum_{l<i} L(i,l) (w_j)_l,
//   w_j <- w_j - U_j Tt_j^t v,
// where s_i = Omega u_i and L(i, l) = s_i . Omega e_l is the strictly lower
// part of (Omega U)^t Omega restricted to the first m columns (the form the
// section gives for operators applied as products).  The sketches E = Omega
// e_l (l < m) of the first m unit vectors are formed once.  The refreshed
// column is sketched (one pass over its n rows, fused with the refresh for a
// Gaussian operator), and trimRHVector needs nothing else:
//   Omega w' = Omega w - E_{<j} w_{<j},  rho = ||Omega w'||,  sigma = sign(w_j),
//   s = Omega w' + sigma rho E_j,  u = (0_j; w_{j:}) + sigma rho e_j, scaled.
// T (right-wise products, eq. Tqdefbis) and Tt (left-wise, eq. Sqdefbis) take
//   t_{<j,j}  = -beta_j T  S_{<j}^t s_j,
//   tt_{<j,j} = -beta_j Tt ([0 Omega_{j:n}] U_{<j})^t s_j
//             = -beta_j Tt (S_{<j}^t s_j - U_top^t (E_{<j}^t s_j)).
// Q = (I - U T ut((Omega U)^t Omega)) [I_m; 0] = [I_m; 0] - U (T ut(S^t E)).
//
// A Gaussian Omega_full = G / sqrt(k) does not have unit columns; its first m
// columns are normalised (Omega' = Omega_full with E_l = G e_l / ||G e_l||),
// and every sketch of x is corrected on the small side:
// Omega' x = Omega_full x + sum_{l<m} E_l (1 - ||Omega_full e_l||) x_l.
// The SRHT has unit columns by construction (k entries +-1/sqrt(k)).
#include "apply.cuh"
#include "column.cuh"
#include "common.cuh"
#include "small.cuh"
#include "trim.cuh"

namespace rhqr {

// E[:, l] = Omega_full e_l for an SRHT: (1/sqrt k) D_l (-1)^{popcount(row_r & l)}
static __global__ void trim_e_srht_kernel(const uint32_t *sign_bits, const int32_t *rows, int32_t k, int32_t m,
                                          double *E, double *nrm) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)k * m) return;
  const int l = (int)(e / k), r = (int)(e - (int64_t)l * k);
  const bool neg = (((sign_bits[l >> 5] >> (l & 31)) & 1u) != 0) ^ ((__popc(rows[r] & l) & 1) != 0);
  E[e] = (neg ? -1.0 : 1.0) / sqrt((double)k);
  if (r == 0) nrm[l] = 1.0;
}

// E[:, l] = G e_l / ||G e_l|| (normalised first m columns of a Gaussian
// Omega_full, stored row-major k x n with ld ldg), nrm[l] = ||G e_l|| / sqrt k.
template <class TG>
static __global__ void trim_e_gauss_kernel(const TG *G, int64_t ldg, int32_t k, double *E, double *nrm) {
  __shared__ double red[32];
  const int l = blockIdx.x;
  double acc = 0.0;
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    const double g = to_f64<TG>(G[(int64_t)r * ldg + l]);
    acc += g * g;
  }
  acc = block_sum(acc, red);
  const double gn = sqrt(acc);
  for (int r = threadIdx.x; r < k; r += blockDim.x) E[(int64_t)l * k + r] = to_f64<TG>(G[(int64_t)r * ldg + l]) / gn;
  if (threadIdx.x == 0) nrm[l] = gn / sqrt((double)k);
}

// Z[:, c] += sum_{l<m} E_l (1 - nrm_l) X[l, c] (the Gaussian correction to
// Omega' of a batch of sketches; X: the batch's top rows, ld ldx)
template <class T>
static __global__ void trim_correct_kernel(double *Z, int64_t ldz, int32_t k, int32_t m, const double *E,
                                           const double *nrm, const T *X, int64_t ldx) {
  const int c = blockIdx.x;
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    double acc = 0.0;
    for (int l = 0; l < m; ++l) acc += E[(int64_t)l * k + r] * ((1.0 - nrm[l]) * (double)X[(int64_t)c * ldx + l]);
    Z[(int64_t)c * ldz + r] += acc;
  }
}

// Step j >= 1: v_i = s_i . z - sum_{l<i} L(i,l) x_l (i < j; z = Omega' w_j,
// x = the top rows of the input column w_j), then c = Tt_j^t v.
static __global__ void trim_coef_kernel(const double *S, int64_t lds, int32_t k, int32_t j, const double *z,
                                        const double *L, int32_t m, const double *x, const double *Tt, double *c) {
  __shared__ double v[1024];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wid; i < j; i += nw) {
    const double *si = S + (int64_t)i * lds;
    double acc = 0.0;
    for (int r = lane; r < k; r += 32) acc += si[r] * z[r];
    acc = warp_sum(acc);
    double low = 0.0;
    for (int l = lane; l < i; l += 32) low += L[(int64_t)l * m + i] * x[l];
    low = warp_sum(low);
    if (lane == 0) v[i] = acc - low;
  }
  __syncthreads();
  // c_t = sum_{i<=t} Tt(i, t) v_i: one warp per t, lanes reading column t (coalesced)
  for (int t = wid; t < j; t += nw) {
    double acc = 0.0;
    for (int i = lane; i <= t; i += 32) acc += Tt[(int64_t)t * m + i] * v[i];
    acc = warp_sum(acc);
    if (lane == 0) c[t] = acc;
  }
}

// trimRHVector at column j: from the sketch zw = Omega_full w of the refreshed
// column and its top rows x (m values): s_j, beta_j, the divisor gamma_j of
// the deferred scaling of u_j, R's column j, the top block of U (scaled, as
// the column kernels will store it) and row j of L.
template <class T>
static __global__ void trim_vector_kernel(const double *zw, const double *E, const double *nrm, int32_t k, int32_t m,
                                          int32_t j, const double *x, int32_t scaling, double *S, int64_t lds,
                                          double *R, double *beta, double *gamma, T *U, int64_t ldu, double *Utop,
                                          double *L, double *zbuf, rhqr_info *info, int *stop) {
  __shared__ double red[32];
  __shared__ double xs[1024];
  if (*stop) return;
  for (int l = threadIdx.x; l < m; l += blockDim.x) xs[l] = x[l];
  __syncthreads();
  const double a = xs[j];
  // Omega' w' = Omega_full w + sum_l E_l (1 - nrm_l) x_l - sum_{l<j} E_l x_l
  double ss = 0.0;
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    double zr = zw[r];
    for (int l = 0; l < m; ++l) {
      const double f = (l < j ? -nrm[l] : 1.0 - nrm[l]) * xs[l];
      zr += E[(int64_t)l * k + r] * f;
    }
    zbuf[r] = zr;
    ss += zr * zr;
  }
  ss = block_sum(ss, red);
  const double rho = sqrt(ss);
  if (!isfinite(rho) || !isfinite(a)) {
    if (threadIdx.x == 0) { set_status(info, RHQR_ENONFINITE, j); *stop = 1; }
    return;
  }
  if (rho == 0.0) {
    if (threadIdx.x == 0) { set_status(info, RHQR_EBREAKDOWN, j); *stop = 1; }
    return;
  }
  const double sigma = a < 0.0 ? -1.0 : 1.0;
  const double g = a + sigma * rho;
  // s = Omega' w' + sigma rho E_j
  double s2 = 0.0;
  for (int r = threadIdx.x; r < k; r += blockDim.x) {
    const double sr = zbuf[r] + sigma * rho * E[(int64_t)j * k + r];
    zbuf[r] = sr;
    s2 += sr * sr;
  }
  s2 = block_sum(s2, red);
  const double div = (scaling == 0) ? g : sqrt(0.5 * s2);
  for (int r = threadIdx.x; r < k; r += blockDim.x) S[(int64_t)j * lds + r] = zbuf[r] / div;
  __syncthreads();
  const T inv_g = (T)(1.0 / div);
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double rv = 0.0, ut = 0.0;
    if (i < j) {
      rv = xs[i];
    } else if (i == j) {
      rv = -sigma * rho;
      ut = scaling == 0 ? 1.0 : (double)((T)g * inv_g);
    } else {
      ut = (double)((T)xs[i] * inv_g);
    }
    R[(int64_t)j * m + i] = i <= j ? rv : 0.0;
    Utop[(int64_t)j * m + i] = ut;
    // top rows of the stored (unscaled) vector: zero above j, g at j
    if (i < j) U[(int64_t)j * ldu + i] = T(0);
    else if (i == j) U[(int64_t)j * ldu + i] = (T)g;
  }
  // row j of L: s_j . E_l (l < j)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int l = wid; l < j; l += nw) {
    double acc = 0.0;
    for (int r = lane; r < k; r += 32) acc += S[(int64_t)j * lds + r] * E[(int64_t)l * k + r];
    acc = warp_sum(acc);
    if (lane == 0) L[(int64_t)l * m + j] = acc;
  }
  if (threadIdx.x == 0) {
    beta[j] = (scaling == 0) ? 2.0 * g * g / s2 : 1.0;
    gamma[j] = div;
  }
}

// Column j of T and Tt (eqs. Tqdefbis, Sqdefbis), diagonals beta_j.
static __global__ void trim_tcol_kernel(const double *S, int64_t lds, int32_t k, int32_t m, int32_t j,
                                        const double *beta, const double *Utop, const double *L, double *T,
                                        double *Tt, const int *stop) {
  __shared__ double d1[1024], d2[1024];
  if (*stop) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int l = wid; l < j; l += nw) {
    double acc = 0.0;
    for (int r = lane; r < k; r += 32) acc += S[(int64_t)l * lds + r] * S[(int64_t)j * lds + r];
    acc = warp_sum(acc);
    if (lane == 0) d1[l] = acc;
  }
  __syncthreads();
  // d2_l = d1_l - sum_{i<j} Utop(i, l) L(j, i)   (Utop(i, l) = 0 for i < l)
  for (int l = wid; l < j; l += nw) {  // one warp per l, lanes over i (Utop column l, coalesced)
    double acc = 0.0;
    for (int i = l + lane; i < j; i += 32) acc += Utop[(int64_t)l * m + i] * L[(int64_t)i * m + j];
    acc = warp_sum(acc);
    if (lane == 0) d2[l] = d1[l] - acc;
  }
  __syncthreads();
  const double bj = beta[j];
  // one warp per row i, lanes over l, fixed-order warp trees
  for (int i = wid; i < m; i += nw) {
    double tv = 0.0, ttv = 0.0;
    if (i < j) {
      for (int l = i + lane; l < j; l += 32) {
        tv += T[(int64_t)l * m + i] * d1[l];
        ttv += Tt[(int64_t)l * m + i] * d2[l];
      }
      tv = -bj * warp_sum(tv);
      ttv = -bj * warp_sum(ttv);
    } else if (i == j) {
      tv = bj;
      ttv = bj;
    }
    if (lane == 0) {
      T[(int64_t)j * m + i] = tv;
      Tt[(int64_t)j * m + i] = ttv;
    }
  }
}

// Gm = T ut(S^t E): Gm(i, c) = sum_{l=i..c} T(i, l) (s_l . E_c), upper triangular.
static __global__ void trim_g_kernel(const double *T, const double *S, int64_t lds, int32_t k, int32_t m,
                                     const double *E, double *Gm) {
  __shared__ double p[1024];
  const int c = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int l = wid; l <= c; l += nw) {
    double acc = 0.0;
    for (int r = lane; r < k; r += 32) acc += S[(int64_t)l * lds + r] * E[(int64_t)c * k + r];
    acc = warp_sum(acc);
    if (lane == 0) p[l] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double acc = 0.0;
    if (i <= c)
      for (int l = i; l <= c; ++l) acc += T[(int64_t)l * m + i] * p[l];
    Gm[(int64_t)c * m + i] = acc;
  }
}

template <class T>
static __global__ void to_f64_kernel(const T *A, int64_t count, double *B) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) B[e] = (double)A[e];
}

size_t trim_workspace_bytes(const SketchView &s, int64_t n, int32_t m, int32_t wt) {
  Carver c(nullptr, 0);
  const int32_t k = s.k;
  c.take<double>((size_t)k * m);  // E
  c.take<double>(m);              // nrm
  c.take<double>((size_t)k * m);  // Zraw
  c.take<double>(k);              // zw
  c.take<double>(k);              // zbuf
  c.take<double>(m);              // x (top rows of the refreshed column)
  c.take<double>((size_t)m * m);  // top rows of the input
  c.take<double>((size_t)m * m);  // L
  c.take<double>((size_t)m * m);  // Utop
  c.take<double>(4 * (size_t)m);  // c, gamma, beta, spare
  c.take<int>(4);
  c.take<double>((size_t)m * m);  // Gm
  c.take<char>(small_padded_bytes(m));
  c.take<char>((size_t)m * m * dtype_size(wt));  // top rows of W in its dtype
  if (s.kind == RHQR_SKETCH_SRHT) c.take<char>((size_t)s.N1 * s.d2 * dtype_size(wt));
  else c.take<double>((size_t)ceil_div(n, LG_RB) * k);
  c.take<char>(sketch_apply_workspace_bytes(s, 0, wt, n, m));
  return c.used() + 1024;
}

template <class T>
static rhqr_status trim_typed(const SketchView &s, const T *W, int64_t n, int32_t m, int64_t ldw, int32_t scaling,
                              T *U, int64_t ldu, double *S, int64_t lds, double *Tm, double *Tt, double *R, T *Q,
                              int64_t ldq, void *ws, size_t ws_bytes, rhqr_info *info, cudaStream_t st) {
  const int32_t k = s.k;
  const int32_t wt = sizeof(T) == 8 ? RHQR_F64 : RHQR_F32;
  Carver cv(ws, ws_bytes);
  double *E = cv.take<double>((size_t)k * m);
  double *nrm = cv.take<double>(m);
  double *Zraw = cv.take<double>((size_t)k * m);
  double *zw = cv.take<double>(k);
  double *zbuf = cv.take<double>(k);
  double *x = cv.take<double>(m);
  double *xin = cv.take<double>((size_t)m * m);
  double *L = cv.take<double>((size_t)m * m);
  double *Utop = cv.take<double>((size_t)m * m);
  double *cbuf = cv.take<double>(m);
  double *gam = cv.take<double>(m);
  double *beta = cv.take<double>(m);
  (void)cv.take<double>(m);
  int *stop = cv.take<int>(4);
  double *Gm = cv.take<double>((size_t)m * m);
  char *GT = cv.take<char>(small_padded_bytes(m));
  T *Wtop = cv.take<T>((size_t)m * m);
  void *stage = nullptr;
  if (s.kind == RHQR_SKETCH_SRHT) stage = cv.take<char>((size_t)s.N1 * s.d2 * sizeof(T));
  else stage = cv.take<double>((size_t)ceil_div(n, LG_RB) * k);
  const size_t apply_ws = sketch_apply_workspace_bytes(s, 0, wt, n, m);
  char *aws = cv.take<char>(apply_ws);
  if (cv.overflow()) return RHQR_ENOMEM;

  RHQR_CUDA_TRY(cudaMemsetAsync(stop, 0, 4 * sizeof(int), st));
  RHQR_CUDA_TRY(cudaMemsetAsync(Tm, 0, sizeof(double) * m * m, st));
  RHQR_CUDA_TRY(cudaMemsetAsync(Tt, 0, sizeof(double) * m * m, st));
  RHQR_CUDA_TRY(cudaMemsetAsync(L, 0, sizeof(double) * m * m, st));
  // E = Omega' e_l (l < m)
  if (s.kind == RHQR_SKETCH_SRHT) {
    trim_e_srht_kernel<<<(unsigned)ceil_div((int64_t)k * m, 256), 256, 0, st>>>(s.sign_bits, s.rows, k, m, E, nrm);
  } else {
    switch (s.omega_dtype) {
      case RHQR_F64: trim_e_gauss_kernel<double><<<m, 256, 0, st>>>((const double *)s.G, s.ldg, k, E, nrm); break;
      case RHQR_F32: trim_e_gauss_kernel<float><<<m, 256, 0, st>>>((const float *)s.G, s.ldg, k, E, nrm); break;
      case RHQR_BF16:
        trim_e_gauss_kernel<__nv_bfloat16><<<m, 256, 0, st>>>((const __nv_bfloat16 *)s.G, s.ldg, k, E, nrm);
        break;
      case RHQR_F16: trim_e_gauss_kernel<__half><<<m, 256, 0, st>>>((const __half *)s.G, s.ldg, k, E, nrm); break;
      default: return RHQR_EINVAL;
    }
  }
  RHQR_LAUNCH_CHECK();
  // raw sketches Omega' w_j of every input column, and the input's top rows
  RHQR_TRY(sketch_apply_simt(s, 0, W, wt, n, m, ldw, Zraw, k, aws, apply_ws, st));
  RHQR_CUDA_TRY(cudaMemcpy2DAsync(Wtop, (size_t)m * sizeof(T), W, (size_t)ldw * sizeof(T), (size_t)m * sizeof(T),
                                  (size_t)m, cudaMemcpyDeviceToDevice, st));
  if (s.kind == RHQR_SKETCH_GAUSSIAN) {
    trim_correct_kernel<T><<<m, 256, 0, st>>>(Zraw, k, k, m, E, nrm, Wtop, m);
    RHQR_LAUNCH_CHECK();
  }
  to_f64_kernel<T><<<(unsigned)ceil_div((int64_t)m * m, 256), 256, 0, st>>>(Wtop, (int64_t)m * m, xin);
  RHQR_LAUNCH_CHECK();

  const double scale = 1.0 / sqrt((double)k);
  // the column kernels copy the refreshed column's top m rows to x and sketch all rows
  ColArgs ca{W, ldw, U, ldu, n, m, 0, cbuf, gam, x, scaling == 0 ? 1 : 0, 0, 0};
  for (int32_t j = 0; j < m; ++j) {
    if (j >= 1) {
      trim_coef_kernel<<<1, 1024, 0, st>>>(S, lds, k, j, Zraw + (int64_t)j * k, L, m, xin + (int64_t)j * m, Tt, cbuf);
      RHQR_LAUNCH_CHECK();
    }
    ca.j = j;
    if (s.kind == RHQR_SKETCH_SRHT) {
      RHQR_TRY(launch_refresh<T>(ca, 1, st));
      RHQR_TRY(column_srht<T>(ca, s, (T *)stage, 1, st));
      left_srht_combine_kernel<T><<<(unsigned)ceil_div(k, 8), 256, 0, st>>>(
          (const T *)stage, s.N1, s.d2, s.sample_i1, s.sample_slot, k, 0, scale, zw);
      RHQR_LAUNCH_CHECK();
    } else {
      const int nbk = (int)ceil_div(n, LG_RB);
      switch (s.omega_dtype) {
        case RHQR_F64:
          left_column_gauss_kernel<T, double><<<nbk, LG_RB, 0, st>>>(ca, (const double *)s.G, s.ldg, k,
                                                                     (double *)stage);
          break;
        case RHQR_F32:
          left_column_gauss_kernel<T, float><<<nbk, LG_RB, 0, st>>>(ca, (const float *)s.G, s.ldg, k,
                                                                    (double *)stage);
          break;
        case RHQR_BF16:
          left_column_gauss_kernel<T, __nv_bfloat16><<<nbk, LG_RB, 0, st>>>(ca, (const __nv_bfloat16 *)s.G, s.ldg,
                                                                            k, (double *)stage);
          break;
        default:
          left_column_gauss_kernel<T, __half><<<nbk, LG_RB, 0, st>>>(ca, (const __half *)s.G, s.ldg, k,
                                                                     (double *)stage);
          break;
      }
      RHQR_LAUNCH_CHECK();
      left_gauss_reduce_kernel<<<(unsigned)ceil_div(k, 128), 128, 0, st>>>((const double *)stage, nbk, k, 0, scale,
                                                                           zw);
      RHQR_LAUNCH_CHECK();
    }
    trim_vector_kernel<T><<<1, 256, 0, st>>>(zw, E, nrm, k, m, j, x, scaling, S, lds, R, beta, gam, U, ldu, Utop, L,
                                             zbuf, info, stop);
    RHQR_LAUNCH_CHECK();
    trim_tcol_kernel<<<1, 1024, 0, st>>>(S, lds, k, m, j, beta, Utop, L, Tm, Tt, stop);
    RHQR_LAUNCH_CHECK();
  }
  left_scale_last_kernel<T><<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(U, ldu, n, m - 1, gam, scaling == 0);
  RHQR_LAUNCH_CHECK();
  if (Q != nullptr) {
    trim_g_kernel<<<m, 256, 0, st>>>(Tm, S, lds, k, m, E, Gm);
    RHQR_LAUNCH_CHECK();
    // (the row pass: G's diagonal beta_j (s_j . E_j) has no bound away from zero,
    // which the tensor-core product with -G would need)
    RHQR_TRY(pad_transpose<T>(Gm, m, 1, (T *)GT, st));
    RHQR_TRY(rows_form_q<T>(U, ldu, 0, n, m, (const T *)GT, Q, ldq, st));
  }
  return RHQR_OK;
}

rhqr_status trim_factor(const SketchView &s, const void *W, int32_t wt, int64_t n, int32_t m, int64_t ldw,
                        int32_t scaling, void *U, int64_t ldu, double *S, int64_t lds, double *T, double *Tt,
                        double *R, void *Q, int64_t ldq, void *ws, size_t ws_bytes, rhqr_info *info,
                        cudaStream_t st) {
  if (wt == RHQR_F64)
    return trim_typed<double>(s, (const double *)W, n, m, ldw, scaling, (double *)U, ldu, S, lds, T, Tt, R,
                              (double *)Q, ldq, ws, ws_bytes, info, st);
  if (wt == RHQR_F32)
    return trim_typed<float>(s, (const float *)W, n, m, ldw, scaling, (float *)U, ldu, S, lds, T, Tt, R, (float *)Q,
                             ldq, ws, ws_bytes, info, st);
  return RHQR_ENOTSUP;
}

}  // namespace rhqr

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
namespace rhqr {
const SketchView *sketch_view_of(rhqr_sketch s);
}
using namespace rhqr;

static rhqr_status trim_check(rhqr_sketch s, int32_t wt, int64_t n, int32_t m) {
  if (s == nullptr || (wt != RHQR_F64 && wt != RHQR_F32) || m < 1 || n <= m) return RHQR_EINVAL;
  const SketchView &v = *sketch_view_of(s);
  if (m > 1024 || (v.kind == RHQR_SKETCH_GAUSSIAN && n != v.n) || (v.kind == RHQR_SKETCH_SRHT && n > v.N))
    return RHQR_EINVAL;
  return RHQR_OK;
}

extern "C" rhqr_status rhqr_trim_workspace(rhqr_sketch s, int32_t wt, int64_t n, int32_t m, size_t *bytes) {
  if (bytes == nullptr) return RHQR_EINVAL;
  RHQR_TRY(trim_check(s, wt, n, m));
  *bytes = trim_workspace_bytes(*sketch_view_of(s), n, m, wt);
  return RHQR_OK;
}

extern "C" rhqr_status rhqr_trim_factor(rhqr_sketch s, const void *W, int32_t wt, int64_t n, int32_t m, int64_t ldw,
                                        int32_t scaling, void *U, int64_t ldu, double *S, int64_t lds, double *T,
                                        double *Tt, double *R, void *Q, int64_t ldq, void *ws, size_t ws_bytes,
                                        rhqr_info *info, rhqr_stream_t stream) {
  RHQR_TRY(trim_check(s, wt, n, m));
  const SketchView &v = *sketch_view_of(s);
  if (W == nullptr || U == nullptr || S == nullptr || T == nullptr || Tt == nullptr || R == nullptr ||
      info == nullptr)
    return RHQR_EINVAL;
  if (ldw < n || ldu < n || lds < v.k || (Q != nullptr && ldq < n) || (scaling != 0 && scaling != 1))
    return RHQR_EINVAL;
  if (ws == nullptr || ws_bytes < trim_workspace_bytes(v, n, m, wt)) return RHQR_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  RHQR_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(rhqr_info), st));
  return trim_factor(v, W, wt, n, m, ldw, scaling, U, ldu, S, lds, T, Tt, R, Q, ldq, ws, ws_bytes, info, st);
}
