// Left-looking RHQR (Algorithm 4) on the GPU.
//
// The raw sketches z_j = Psi w_j of all columns are formed once up front (the
// sketch of column j taken at the start of step j only depends on the
// untouched input column).  Step j then runs:
//   1. c = T_j^t (S_j^t z_j)                               (small, float64)
//   2. column kernel: w_j <- w_j - U_{:, <j} c over all n rows, written to
//      U[:, j]; the previous column's deferred scale u_{j-1} = u~_{j-1}/gamma
//      is applied while it is read (and written back); the refreshed column
//      is sketched in the same pass (SRHT stage A on the block's rows, or the
//      Gaussian partial products); rows < m are copied into y exactly
//   3. y = Psi w_j (SRHT stage B / ordered reduction of Gaussian partials)
//   4. RHVector (Algorithm 2) on (w_j, y): sigma, rho, gamma, beta, s_j, r_j
//   5. t_j = (-beta T_j S_j^t s_j; beta) and the next step's coefficients.
#include "apply.cuh"
#include "column.cuh"
#include "common.cuh"
#include "left.cuh"
#include "small.cuh"

namespace rhqr {

// ---------------------------------------------------------------------------
// step 1 / 5 helpers
// dots over the columns l = lo + t of the current block (lo = 0: all previous
// columns): d[t] = S[:, l] . s_j (t < nd), v[t] = S[:, l] . z (t < nv)
// ---------------------------------------------------------------------------
__global__ void left_dots_kernel(const double *S, int64_t lds, int64_t p, int32_t j, int32_t nd, const double *z,
                                 int32_t nv, double *d, double *v, int32_t lo, int64_t bs_S = 0, int64_t bs_z = 0,
                                 int64_t bs_vec = 0) {
  pdl_wait();
  pdl_release();
  __shared__ double red[32];
  S += (int64_t)blockIdx.z * bs_S;  // problem blockIdx.z of a batch
  z += (int64_t)blockIdx.z * bs_z;
  d += (int64_t)blockIdx.z * bs_vec;
  v += (int64_t)blockIdx.z * bs_vec;
  const int t = blockIdx.x;  // d[t], v[t] belong to column l = lo + t
  const int l = lo + t;
  int which = blockIdx.y;  // 0: d (against s_j), 1: v (against z)
  if ((which == 0 && t >= nd) || (which == 1 && t >= nv)) return;
  const double *a = S + (int64_t)l * lds;
  const double *b = (which == 0) ? S + (int64_t)j * lds : z;
  int64_t start = (which == 0) ? j : l;  // s_j vanishes above j, s_l above l
  double acc = 0.0;
  for (int64_t r = start + threadIdx.x; r < p; r += blockDim.x) acc += a[r] * b[r];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) {
    if (which == 0) d[t] = acc;
    else v[t] = acc;
  }
}

// Within the block of columns lo, lo + 1, ... (lo = 0: one block of all
// columns): T[:, j] from d (if j >= 0, finishing column j; rows above lo are
// zero, the block's T is a diagonal block), then c = T_blk^t v for the nc
// block columns lo .. lo + nc - 1.
__global__ void left_tcol_coef_kernel(double *T, int32_t m, int32_t j, const double *beta, const double *d,
                                      const double *v, int32_t nc, double *c, int32_t lo, int64_t bs_T = 0,
                                      int64_t bs_vec = 0) {
  pdl_wait();
  pdl_release();
  T += (int64_t)blockIdx.x * bs_T;  // problem blockIdx.x of a batch (one block each)
  beta += (int64_t)blockIdx.x * bs_vec;
  d += (int64_t)blockIdx.x * bs_vec;
  v += (int64_t)blockIdx.x * bs_vec;
  c += (int64_t)blockIdx.x * bs_vec;
  if (j >= 0) {
    // t_i = -beta_j sum_{l=i}^{j-1} T(i, l) d_l: one warp per row i, lanes over
    // l (the loads of all warps in flight together), fixed-order warp tree
    const double bj = beta[j];
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = threadIdx.x >> 5; i < m; i += nw) {
      double val = 0.0;
      if (i >= lo && i < j) {
        double acc = 0.0;
        for (int l = i + lane; l < j; l += 32) acc += T[(int64_t)l * m + i] * d[l - lo];
        val = -bj * warp_sum(acc);
      } else if (i == j) {
        val = bj;
      }
      if (lane == 0) T[(int64_t)j * m + i] = val;
    }
    __syncthreads();
  }
  // c_t = sum_{i=lo}^{l} T(i, l) v_{i-lo}, l = lo + t: one warp per t, the
  // lanes reading column l of T (coalesced), fixed-order warp tree
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = threadIdx.x >> 5; t < nc; t += nw) {
    const int l = lo + t;
    double acc = 0.0;
    for (int i = lo + lane; i <= l; i += 32) acc += T[(int64_t)l * m + i] * v[i - lo];
    acc = warp_sum(acc);
    if (lane == 0) c[t] = acc;
  }
}

// ---------------------------------------------------------------------------
// step 4: RHVector on y (Algorithm 2), one block
// ---------------------------------------------------------------------------
// Batches: problem blockIdx.x (one block each), element strides bs_*.
struct RhvBatch {
  int64_t y, S, R, vec, U, stop;
};

template <class T>
__global__ void left_rhvector_kernel(const double *y, int64_t p, int32_t m, int32_t j, int32_t scaling, double *S,
                                     int64_t lds, double *R, double *beta, double *gamma_out, T *U, int64_t ldu,
                                     rhqr_info *info, int *stop, RhvBatch bb = RhvBatch{}) {
  pdl_wait();
  pdl_release();
  __shared__ double red[32];
  {
    const int64_t b = blockIdx.x;
    y += b * bb.y;
    S += b * bb.S;
    R += b * bb.R;
    beta += b * bb.vec;
    gamma_out += b * bb.vec;
    U += b * bb.U;
    stop += b * bb.stop;
    if (info != nullptr) info += b;
  }
  if (*stop) return;
  double s = 0.0;
  for (int64_t r = j + threadIdx.x; r < p; r += blockDim.x) s += y[r] * y[r];
  s = block_sum(s, red);
  const double rho = sqrt(s);
  const double a = y[j];
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
  const double div = (scaling == 0) ? g : sqrt(rho * (rho + fabs(a)));
  for (int64_t r = threadIdx.x; r < p; r += blockDim.x) {
    double v = 0.0;
    if (r == j) v = g / div;
    else if (r > j) v = y[r] / div;
    S[(int64_t)j * lds + r] = v;
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double rv = 0.0;
    if (i < j) rv = y[i];
    else if (i == j) rv = -sigma * rho;
    R[(int64_t)j * m + i] = rv;
    // top rows of the stored vector: zero above j, gamma (unscaled) at j
    if (i < j) U[(int64_t)j * ldu + i] = T(0);
    else if (i == j) U[(int64_t)j * ldu + i] = (T)g;
  }
  if (threadIdx.x == 0) {
    beta[j] = (scaling == 0) ? 1.0 + fabs(a) / rho : 1.0;
    gamma_out[j] = div;
  }
}

// ---------------------------------------------------------------------------
// host
// ---------------------------------------------------------------------------

size_t left_workspace_bytes(const SketchView &s, int64_t n, int32_t m, int32_t wt) {
  Carver c(nullptr, 0);
  int64_t p = (int64_t)s.k + m;
  c.take<double>((size_t)p * m);  // Zraw
  c.take<double>(p);              // y
  c.take<double>(4 * (size_t)m);  // c, v, d, gamma
  c.take<double>(m);              // beta
  c.take<int>(4);                 // stop flag
  c.take<double>((size_t)m * m);  // G = T U_1^t
  c.take<char>(small_padded_bytes(m));
  if (s.kind == RHQR_SKETCH_SRHT) c.take<char>((size_t)s.N1 * s.d2 * dtype_size(wt));
  else c.take<double>((size_t)ceil_div(n, LG_RB) * s.k);
  size_t apply_ws = sketch_apply_workspace_bytes(s, m, wt, n, m);
  return c.used() + align_up(apply_ws, 256) + 1024;
}

template <class T>
static rhqr_status left_typed(const SketchView &s, const T *W, int64_t n, int32_t m, int64_t ldw, int32_t scaling,
                              T *U, int64_t ldu, double *S, int64_t lds, double *Tm, double *R, T *Q, int64_t ldq,
                              void *ws, size_t ws_bytes, rhqr_info *info, cudaStream_t st) {
  const int64_t p = (int64_t)s.k + m;
  Carver cv(ws, ws_bytes);
  double *Zraw = cv.take<double>((size_t)p * m);
  double *y = cv.take<double>(p);
  double *cbuf = cv.take<double>(m);
  double *vbuf = cv.take<double>(m);
  double *dbuf = cv.take<double>(m);
  double *gam = cv.take<double>(m);
  double *beta = cv.take<double>(m);
  int *stop = cv.take<int>(4);
  double *Gm = cv.take<double>((size_t)m * m);
  char *GT = cv.take<char>(small_padded_bytes(m));
  void *stage = nullptr;
  if (s.kind == RHQR_SKETCH_SRHT) stage = cv.take<char>((size_t)s.N1 * s.d2 * sizeof(T));
  else stage = cv.take<double>((size_t)ceil_div(n, LG_RB) * s.k);
  size_t apply_ws = sketch_apply_workspace_bytes(s, m, sizeof(T) == 8 ? RHQR_F64 : RHQR_F32, n, m);
  char *aws = cv.take<char>(apply_ws);
  if (cv.overflow()) return RHQR_ENOMEM;
  if (m > 1024) return RHQR_ENOTSUP;

  RHQR_CUDA_TRY(cudaMemsetAsync(stop, 0, 4 * sizeof(int), st));
  RHQR_CUDA_TRY(cudaMemsetAsync(Tm, 0, sizeof(double) * m * m, st));
  // raw sketches of all columns (Algorithm 4 sketches w_j before refreshing it)
  RHQR_TRY(sketch_apply_simt(s, m, W, sizeof(T) == 8 ? RHQR_F64 : RHQR_F32, n, m, ldw, Zraw, p, aws, apply_ws, st));

  ColArgs ca{W, ldw, U, ldu, n, m, 0, cbuf, gam, y, scaling == 0 ? 1 : 0, 0, m};
  const double scale = 1.0 / sqrt((double)s.k);
  for (int j = 0; j < m; ++j) {
    if (j >= 1) {
      // d_l = s_l . s_{j-1} (l < j-1) finishes column j-1 of T; v_l = s_l . z_j (l < j)
      // the chain of each column is launched with PDL (launch_pdl): each kernel
      // is scheduled while its predecessor runs and waits for it on the device
      dim3 g((unsigned)j, 2);
      RHQR_CUDA_TRY(launch_pdl(left_dots_kernel, g, dim3(256), 0, st, (const double *)S, lds, p, j - 1, j - 1,
                               (const double *)(Zraw + (int64_t)j * p), j, dbuf, vbuf, 0, (int64_t)0, (int64_t)0,
                               (int64_t)0));
      RHQR_LAUNCH_CHECK();
      RHQR_CUDA_TRY(launch_pdl(left_tcol_coef_kernel, dim3(1), dim3(1024), 0, st, Tm, m, j - 1, (const double *)beta,
                               (const double *)dbuf, (const double *)vbuf, j, cbuf, 0, (int64_t)0, (int64_t)0));
      RHQR_LAUNCH_CHECK();
    }
    ca.j = j;
    if (s.kind == RHQR_SKETCH_SRHT) {
      // refresh with the whole GPU, then sign / transform / sample the refreshed column
      RHQR_TRY(launch_refresh<T>(ca, 1, st));
      RHQR_TRY(column_srht<T>(ca, s, (T *)stage, 1, st));
      RHQR_CUDA_TRY(launch_pdl(left_srht_combine_kernel<T>, dim3((unsigned)ceil_div(s.k, 8)), dim3(256), 0, st,
                               (const T *)stage, s.N1, s.d2, s.sample_i1, s.sample_slot, s.k, m, scale, y,
                               (int64_t)0, (int64_t)0));
      RHQR_LAUNCH_CHECK();
    } else {
      int nb = (int)ceil_div(n, LG_RB);
      switch (s.omega_dtype) {
        case RHQR_F64:
          left_column_gauss_kernel<T, double><<<nb, LG_RB, 0, st>>>(ca, (const double *)s.G, s.ldg, s.k,
                                                                    (double *)stage);
          break;
        case RHQR_F32:
          left_column_gauss_kernel<T, float><<<nb, LG_RB, 0, st>>>(ca, (const float *)s.G, s.ldg, s.k,
                                                                   (double *)stage);
          break;
        case RHQR_BF16:
          left_column_gauss_kernel<T, __nv_bfloat16><<<nb, LG_RB, 0, st>>>(ca, (const __nv_bfloat16 *)s.G, s.ldg,
                                                                           s.k, (double *)stage);
          break;
        case RHQR_F16:
          left_column_gauss_kernel<T, __half><<<nb, LG_RB, 0, st>>>(ca, (const __half *)s.G, s.ldg, s.k,
                                                                    (double *)stage);
          break;
        default:
          return RHQR_EINVAL;
      }
      RHQR_LAUNCH_CHECK();
      left_gauss_reduce_kernel<<<(unsigned)ceil_div(s.k, 128), 128, 0, st>>>((const double *)stage, nb, s.k, m,
                                                                             scale, y);
      RHQR_LAUNCH_CHECK();
    }
    RHQR_CUDA_TRY(launch_pdl(left_rhvector_kernel<T>, dim3(1), dim3(256), 0, st, (const double *)y, p, m, j, scaling,
                             S, lds, R, beta, gam, U, ldu, info, stop, RhvBatch{}));
    RHQR_LAUNCH_CHECK();
  }
  // finish T's last column and the last column's scale
  {
    dim3 g((unsigned)std::max(1, m - 1), 2);
    left_dots_kernel<<<g, 256, 0, st>>>(S, lds, p, m - 1, m - 1, Zraw, 0, dbuf, vbuf, 0);
    RHQR_LAUNCH_CHECK();
    left_tcol_coef_kernel<<<1, 1024, 0, st>>>(Tm, m, m - 1, beta, dbuf, vbuf, 0, cbuf, 0);
    RHQR_LAUNCH_CHECK();
    left_scale_last_kernel<T><<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(U, ldu, n, m - 1, gam, scaling == 0);
    RHQR_LAUNCH_CHECK();
  }
  if (Q != nullptr) {
    // Q = [I; 0] - U (T U_1^t)  (Section 3.2)
    RHQR_TRY(t_u1t(Tm, S, lds, m, Gm, st));
    RHQR_TRY(form_q_from_g<T>(U, ldu, n, m, Gm, GT, Q, ldq, info, st));
  }
  return RHQR_OK;
}

rhqr_status left_factor(const SketchView &s, const void *W, int32_t wt, int64_t n, int32_t m, int64_t ldw,
                        int32_t scaling, void *U, int64_t ldu, double *S, int64_t lds, double *T, double *R, void *Q,
                        int64_t ldq, void *ws, size_t ws_bytes, rhqr_info *info, cudaStream_t st) {
  if (wt == RHQR_F64)
    return left_typed<double>(s, (const double *)W, n, m, ldw, scaling, (double *)U, ldu, S, lds, T, R,
                              (double *)Q, ldq, ws, ws_bytes, info, st);
  if (wt == RHQR_F32)
    return left_typed<float>(s, (const float *)W, n, m, ldw, scaling, (float *)U, ldu, S, lds, T, R, (float *)Q,
                             ldq, ws, ws_bytes, info, st);
  return RHQR_ENOTSUP;
}

// ---------------------------------------------------------------------------
// blockRHQR (Algorithm 5): the columns in blocks of bs.  Block j is refreshed
// with every earlier block k in turn,
//   Y = Psi W^(j),  C = T^(k)t S^(k)t Y,  W^(j) <- W^(j) - U^(k) C,
// its rows above the block are R's off-diagonal block (they are no longer
// changed), and Algorithm 4 factors it with the global Psi and the global
// column indices, using only the block's own reflectors (lo = first column).
// ---------------------------------------------------------------------------

// C = T_k^t (S_k^t Y) for the kb reflectors of an earlier block starting at
// column k0 (S_k: p x kb, column l vanishing above row k0 + l; T_k: its kb x kb
// upper-triangular diagonal block of T, ld ldt) and the nb columns of Y
// (p x nb, ldy).  C is kb x nb, column-major.  One CTA per column of Y.
__global__ void block_coef_kernel(const double *Sk, int64_t lds, int64_t p, int32_t k0, const double *Tk,
                                  int32_t ldt, int32_t kb, const double *Y, int64_t ldy, double *C) {
  __shared__ double m1[1024];
  const int c = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double *y = Y + (int64_t)c * ldy;
  for (int l = wid; l < kb; l += nw) {
    const double *sl = Sk + (int64_t)l * lds;
    double acc = 0.0;
    for (int64_t r = k0 + l + lane; r < p; r += 32) acc += sl[r] * y[r];
    acc = warp_sum(acc);
    if (lane == 0) m1[l] = acc;
  }
  __syncthreads();
  for (int l = threadIdx.x; l < kb; l += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i <= l; ++i) acc += Tk[(int64_t)l * ldt + i] * m1[i];
    C[(int64_t)c * kb + l] = acc;
  }
}

// Wb[i, c] -= sum_l Uk[i, l] C(l, c) for every row i (one row per thread,
// grid-stride): each row of U_k and of the block is read once and the block's
// row written once; C (kb x nb <= 64 x 64) sits in shared memory.
constexpr int kMaxBlockCols = 64;
template <class T, int NB>
__global__ void __launch_bounds__(256) block_update_kernel(const T *Uk, int64_t ldu, int32_t kb, const double *C,
                                                           T *Wb, int64_t ldw, int32_t nb, int64_t n) {
  __shared__ T Cs[kMaxBlockCols * NB];  // Cs[l * NB + c], zero for c >= nb
  for (int e = threadIdx.x; e < kb * NB; e += blockDim.x) {
    const int l = e / NB, c = e - l * NB;
    Cs[e] = c < nb ? (T)C[(int64_t)c * kb + l] : T(0);
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T acc[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) acc[c] = c < nb ? Wb[(int64_t)c * ldw + i] : T(0);
    for (int l = 0; l < kb; ++l) {
      const T u = Uk[(int64_t)l * ldu + i];
      const T *cl = Cs + l * NB;
#pragma unroll
      for (int c = 0; c < NB; ++c) acc[c] -= u * cl[c];
    }
#pragma unroll
    for (int c = 0; c < NB; ++c)
      if (c < nb) Wb[(int64_t)c * ldw + i] = acc[c];
  }
}

template <class T>
static rhqr_status block_update(const T *Uk, int64_t ldu, int32_t kb, const double *C, T *Wb, int64_t ldw,
                                int32_t nb, int64_t n, cudaStream_t st) {
  const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(n, 256), 152 * 8);
  if (nb <= 16) block_update_kernel<T, 16><<<grid, 256, 0, st>>>(Uk, ldu, kb, C, Wb, ldw, nb, n);
  else if (nb <= 32) block_update_kernel<T, 32><<<grid, 256, 0, st>>>(Uk, ldu, kb, C, Wb, ldw, nb, n);
  else block_update_kernel<T, 64><<<grid, 256, 0, st>>>(Uk, ldu, kb, C, Wb, ldw, nb, n);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

size_t block_workspace_bytes(const SketchView &s, int64_t n, int32_t m, int32_t bs, int32_t wt) {
  Carver c(nullptr, 0);
  c.take<char>(left_workspace_bytes(s, n, m, wt));
  c.take<double>((size_t)kMaxBlockCols * kMaxBlockCols);  // C
  c.take<double>((size_t)m * m);                          // S^t S scratch of the Woodbury T
  (void)bs;
  return c.used() + 1024;
}

template <class T>
static rhqr_status block_typed(const SketchView &s, const T *W, int64_t n, int32_t m, int64_t ldw, int32_t bs,
                               int32_t scaling, T *U, int64_t ldu, double *S, int64_t lds, double *Tm, double *R,
                               T *Q, int64_t ldq, void *ws, size_t ws_bytes, rhqr_info *info, cudaStream_t st) {
  const int64_t p = (int64_t)s.k + m;
  const int32_t wt = sizeof(T) == 8 ? RHQR_F64 : RHQR_F32;
  Carver cv(ws, ws_bytes);
  double *Zraw = cv.take<double>((size_t)p * m);
  double *y = cv.take<double>(p);
  double *cbuf = cv.take<double>(m);
  double *vbuf = cv.take<double>(m);
  double *dbuf = cv.take<double>(m);
  double *gam = cv.take<double>(m);
  double *beta = cv.take<double>(m);
  int *stop = cv.take<int>(4);
  double *Gm = cv.take<double>((size_t)m * m);
  char *GT = cv.take<char>(small_padded_bytes(m));
  void *stage = nullptr;
  if (s.kind == RHQR_SKETCH_SRHT) stage = cv.take<char>((size_t)s.N1 * s.d2 * sizeof(T));
  else stage = cv.take<double>((size_t)ceil_div(n, LG_RB) * s.k);
  const size_t apply_ws = sketch_apply_workspace_bytes(s, m, wt, n, m);
  char *aws = cv.take<char>(apply_ws);
  double *Cb = cv.take<double>((size_t)kMaxBlockCols * kMaxBlockCols);
  double *SS = cv.take<double>((size_t)m * m);
  if (cv.overflow()) return RHQR_ENOMEM;
  if (m > 1024 || bs < 1 || bs > kMaxBlockCols) return RHQR_ENOTSUP;

  RHQR_CUDA_TRY(cudaMemsetAsync(stop, 0, 4 * sizeof(int), st));
  RHQR_CUDA_TRY(cudaMemsetAsync(Tm, 0, sizeof(double) * m * m, st));
  // the blocks are refreshed in place in U
  RHQR_CUDA_TRY(cudaMemcpy2DAsync(U, (size_t)ldu * sizeof(T), W, (size_t)ldw * sizeof(T), (size_t)n * sizeof(T),
                                  (size_t)m, cudaMemcpyDeviceToDevice, st));
  const double scale = 1.0 / sqrt((double)s.k);
  ColArgs ca{U, ldu, U, ldu, n, m, 0, cbuf, gam, y, scaling == 0 ? 1 : 0, 0, m};
  for (int32_t c0 = 0; c0 < m; c0 += bs) {
    const int32_t c1 = std::min(m, c0 + bs), nb = c1 - c0;
    T *Wb = U + (int64_t)c0 * ldu;
    double *Zb = Zraw + (int64_t)c0 * p;
    // refresh with each earlier block in turn, re-sketching the block every time
    for (int32_t k0 = 0; k0 < c0; k0 += bs) {
      const int32_t kb = std::min(bs, c0 - k0);
      RHQR_TRY(sketch_apply_simt(s, m, Wb, wt, n, nb, ldu, Zb, p, aws, apply_ws, st));
      block_coef_kernel<<<(unsigned)nb, 256, 0, st>>>(S + (int64_t)k0 * lds, lds, p, k0, Tm + (int64_t)k0 * m + k0, m,
                                                      kb, Zb, p, Cb);
      RHQR_LAUNCH_CHECK();
      RHQR_TRY(block_update<T>(U + (int64_t)k0 * ldu, ldu, kb, Cb, Wb, ldu, nb, n, st));
    }
    // Algorithm 4 on the refreshed block: raw sketches first
    RHQR_TRY(sketch_apply_simt(s, m, Wb, wt, n, nb, ldu, Zb, p, aws, apply_ws, st));
    ca.lo = c0;
    for (int32_t j = c0; j < c1; ++j) {
      if (j > c0) {
        dim3 g((unsigned)(j - c0), 2);
        left_dots_kernel<<<g, 256, 0, st>>>(S, lds, p, j - 1, j - 1 - c0, Zraw + (int64_t)j * p, j - c0, dbuf, vbuf,
                                            c0);
        RHQR_LAUNCH_CHECK();
        left_tcol_coef_kernel<<<1, 1024, 0, st>>>(Tm, m, j - 1, beta, dbuf, vbuf, j - c0, cbuf, c0);
        RHQR_LAUNCH_CHECK();
      }
      ca.j = j;
      if (s.kind == RHQR_SKETCH_SRHT) {
        RHQR_TRY(launch_refresh<T>(ca, 1, st));
        RHQR_TRY(column_srht<T>(ca, s, (T *)stage, 1, st));
        left_srht_combine_kernel<T><<<(unsigned)ceil_div(s.k, 8), 256, 0, st>>>(
            (const T *)stage, s.N1, s.d2, s.sample_i1, s.sample_slot, s.k, m, scale, y);
        RHQR_LAUNCH_CHECK();
      } else {
        const int nbk = (int)ceil_div(n, LG_RB);
        switch (s.omega_dtype) {
          case RHQR_F64:
            left_column_gauss_kernel<T, double><<<nbk, LG_RB, 0, st>>>(ca, (const double *)s.G, s.ldg, s.k,
                                                                       (double *)stage);
            break;
          case RHQR_F32:
            left_column_gauss_kernel<T, float><<<nbk, LG_RB, 0, st>>>(ca, (const float *)s.G, s.ldg, s.k,
                                                                      (double *)stage);
            break;
          case RHQR_BF16:
            left_column_gauss_kernel<T, __nv_bfloat16><<<nbk, LG_RB, 0, st>>>(ca, (const __nv_bfloat16 *)s.G, s.ldg,
                                                                              s.k, (double *)stage);
            break;
          case RHQR_F16:
            left_column_gauss_kernel<T, __half><<<nbk, LG_RB, 0, st>>>(ca, (const __half *)s.G, s.ldg, s.k,
                                                                       (double *)stage);
            break;
          default:
            return RHQR_EINVAL;
        }
        RHQR_LAUNCH_CHECK();
        left_gauss_reduce_kernel<<<(unsigned)ceil_div(s.k, 128), 128, 0, st>>>((const double *)stage, nbk, s.k, m,
                                                                               scale, y);
        RHQR_LAUNCH_CHECK();
      }
      left_rhvector_kernel<T><<<1, 256, 0, st>>>(y, p, m, j, scaling, S, lds, R, beta, gam, U, ldu, info, stop);
      RHQR_LAUNCH_CHECK();
    }
    // finish the block's T (its last column) and the last column's deferred scale
    {
      dim3 g((unsigned)std::max(1, nb - 1), 2);
      left_dots_kernel<<<g, 256, 0, st>>>(S, lds, p, c1 - 1, nb - 1, Zraw, 0, dbuf, vbuf, c0);
      RHQR_LAUNCH_CHECK();
      left_tcol_coef_kernel<<<1, 1024, 0, st>>>(Tm, m, c1 - 1, beta, dbuf, vbuf, 0, cbuf, c0);
      RHQR_LAUNCH_CHECK();
      left_scale_last_kernel<T><<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(U, ldu, n, c1 - 1, gam, scaling == 0);
      RHQR_LAUNCH_CHECK();
    }
  }
  // the compact form of all m reflectors: T^{-1} = sut(S^t S) + diag(1 / beta)
  // (eq. generalwoodburry); its diagonal blocks are the blocks' T^(j)
  RHQR_TRY(t_factor_small(S, lds, p, m, beta, SS, Tm, st));
  if (Q != nullptr) {
    RHQR_TRY(t_u1t(Tm, S, lds, m, Gm, st));
    RHQR_TRY(form_q_from_g<T>(U, ldu, n, m, Gm, GT, Q, ldq, info, st));
  }
  return RHQR_OK;
}

rhqr_status block_factor(const SketchView &s, const void *W, int32_t wt, int64_t n, int32_t m, int64_t ldw,
                         int32_t bs, int32_t scaling, void *U, int64_t ldu, double *S, int64_t lds, double *T,
                         double *R, void *Q, int64_t ldq, void *ws, size_t ws_bytes, rhqr_info *info,
                         cudaStream_t st) {
  if (wt == RHQR_F64)
    return block_typed<double>(s, (const double *)W, n, m, ldw, bs, scaling, (double *)U, ldu, S, lds, T, R,
                               (double *)Q, ldq, ws, ws_bytes, info, st);
  if (wt == RHQR_F32)
    return block_typed<float>(s, (const float *)W, n, m, ldw, bs, scaling, (float *)U, ldu, S, lds, T, R, (float *)Q,
                              ldq, ws, ws_bytes, info, st);
  return RHQR_ENOTSUP;
}

// ---------------------------------------------------------------------------
// RHQR-Arnoldi (Algorithm 7) on the same kernels, for a batch of nrhs
// independent processes (one per right-hand side) sharing the sketch: every
// kernel of a step is launched once for the whole batch, the process index
// taken from the grid, and each process's arrays lie at a fixed stride.
// ---------------------------------------------------------------------------

// coef_l = sum_{i >= l} T[l, i] S[j, i] for l <= j (x = T_{j+1} S_{j+1}^t e_j),
// the last one divided by gamma_j (column j of U is stored unscaled).  One
// block per process.
__global__ void arnoldi_coef_kernel(const double *T, int32_t M, const double *S, int64_t lds, int32_t j,
                                    const double *gamma, double *coef, int64_t bs_S) {
  pdl_wait();
  pdl_release();
  const int64_t b = blockIdx.x;
  T += b * (int64_t)M * M;
  S += b * bs_S;
  gamma += b * M;
  coef += b * M;
  // one warp per l, lanes over i (fixed-order warp tree)
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int l = threadIdx.x >> 5; l <= j; l += nw) {
    double acc = 0.0;
    for (int i = l + lane; i <= j; i += 32) acc += T[(int64_t)i * M + l] * S[(int64_t)i * lds + j];
    acc = warp_sum(acc);
    if (lane == 0) coef[l] = l == j ? acc / gamma[j] : acc;
  }
}

// q = e_j - U[:, 0..j] coef over all n rows; column j of U is unscaled except
// rows <= j (zeros above, gamma at j), so row j gives exactly 1 - coef_j gamma_j / gamma_j.
// Process blockIdx.y; q of process b at q + b n.
template <class T>
__global__ void arnoldi_q_kernel(const T *U, int64_t ldu, int64_t n, int32_t j, const double *coef, T *q,
                                 int64_t bs_U, int32_t M) {
  const int64_t b = blockIdx.y;
  U += b * bs_U;
  coef += b * M;
  q += b * n;
  __shared__ double c_s[1024];
  for (int l = threadIdx.x; l <= j; l += blockDim.x) c_s[l] = coef[l];
  __syncthreads();
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = (i == j) ? 1.0 : 0.0;
  for (int l = 0; l <= j; ++l) acc -= (double)U[(int64_t)l * ldu + i] * c_s[l];
  q[i] = (T)acc;
}

// Vector form for 16-byte aligned U and q (float32 basis): each thread takes
// V = 16 / sizeof(T) consecutive rows with one 16-byte load per column, four
// independent chains in the basis precision (as the column refresh); the last
// n % V rows go one at a time.
template <class T>
__global__ void __launch_bounds__(256) arnoldi_q_vec_kernel(const T *U, int64_t ldu, int64_t n, int32_t j,
                                                            const double *coef, T *q, int64_t bs_U, int32_t M) {
  pdl_wait();
  using VT = typename Vec16<T>::type;
  constexpr int V = Vec16<T>::V;
  const int64_t b = blockIdx.y;
  U += b * bs_U;
  coef += b * M;
  q += b * n;
  __shared__ T c_s[1024];
  for (int l = threadIdx.x; l <= j; l += blockDim.x) c_s[l] = (T)coef[l];
  __syncthreads();
  const int64_t nvec = n / V;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nvec + (n % V != 0);
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = v * V;
    if (v < nvec) {
      T p[4][V];
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int e = 0; e < V; ++e) p[t][e] = T(0);
      const T *up = U + i0;
      int l = 0;
      for (; l + 4 <= j + 1; l += 4) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const VT u = *reinterpret_cast<const VT *>(up + t * ldu);
          const T *ue = reinterpret_cast<const T *>(&u);
#pragma unroll
          for (int e = 0; e < V; ++e) p[t][e] += ue[e] * c_s[l + t];
        }
        up += 4 * ldu;
      }
      for (; l <= j; ++l, up += ldu) {
        const VT u = *reinterpret_cast<const VT *>(up);
        const T *ue = reinterpret_cast<const T *>(&u);
#pragma unroll
        for (int e = 0; e < V; ++e) p[l & 3][e] += ue[e] * c_s[l];
      }
      VT out;
      T *oe = reinterpret_cast<T *>(&out);
#pragma unroll
      for (int e = 0; e < V; ++e) oe[e] = (i0 + e == j ? T(1) : T(0)) - ((p[0][e] + p[1][e]) + (p[2][e] + p[3][e]));
      *reinterpret_cast<VT *>(q + i0) = out;
    } else {
      for (int64_t i = i0; i < n; ++i) {
        T ps[4] = {T(0), T(0), T(0), T(0)};
        for (int l = 0; l <= j; ++l) ps[l & 3] += U[(int64_t)l * ldu + i] * c_s[l];
        q[i] = (i == j ? T(1) : T(0)) - ((ps[0] + ps[1]) + (ps[2] + ps[3]));
      }
    }
  }
}

static int64_t arnoldi_stage_elems(const SketchView &s, int64_t n) {
  return s.kind == RHQR_SKETCH_SRHT ? (int64_t)s.N1 * s.d2 : ceil_div(n, LG_RB) * s.k;
}

size_t arnoldi_state_bytes(const SketchView &s, int64_t n, int32_t M, int32_t dt, int32_t nrhs) {
  Carver c(nullptr, 0);
  const int64_t p = (int64_t)s.k + M;
  c.take<char>((size_t)n * M * dtype_size(dt) * nrhs);  // U
  c.take<double>((size_t)p * M * nrhs);                  // S
  c.take<double>((size_t)M * M * nrhs);                  // T
  c.take<double>((6 * (size_t)M + 2 * p) * nrhs);        // beta gamma c v d coef; y z
  c.take<int>(4 * (size_t)nrhs);
  const size_t es = s.kind == RHQR_SKETCH_SRHT ? dtype_size(dt) : sizeof(double);
  c.take<char>((size_t)arnoldi_stage_elems(s, n) * es * nrhs);
  c.take<char>(sketch_apply_workspace_bytes(s, M, dt, n, nrhs));
  return c.used() + 1024;
}

rhqr_status arnoldi_carve(ArnoldiState &a, void *mem, size_t bytes) {
  Carver c(mem, bytes);
  const int64_t p = (int64_t)a.view.k + a.M;
  const int32_t B = a.nrhs, M = a.M;
  a.U = c.take<char>((size_t)a.n * M * dtype_size(a.dtype) * B);
  a.ldu = a.n;
  a.S = c.take<double>((size_t)p * M * B);
  a.lds = p;
  a.T = c.take<double>((size_t)M * M * B);
  double *vecs = c.take<double>((6 * (size_t)M + 2 * p) * B);
  a.beta = vecs;
  a.gamma = vecs + (size_t)M * B;
  a.c = vecs + 2 * (size_t)M * B;
  a.v = vecs + 3 * (size_t)M * B;
  a.d = vecs + 4 * (size_t)M * B;
  a.coef = vecs + 5 * (size_t)M * B;
  a.y = vecs + 6 * (size_t)M * B;
  a.z = a.y + (size_t)p * B;
  a.stop = c.take<int>(4 * (size_t)B);
  a.stage_elems = arnoldi_stage_elems(a.view, a.n);
  const size_t es = a.view.kind == RHQR_SKETCH_SRHT ? dtype_size(a.dtype) : sizeof(double);
  a.stage_bytes = (size_t)a.stage_elems * es * B;
  a.stage = c.take<char>(a.stage_bytes);
  a.aws_bytes = sketch_apply_workspace_bytes(a.view, M, a.dtype, a.n, B);
  a.aws = c.take<char>(a.aws_bytes);
  return c.overflow() ? RHQR_ENOMEM : RHQR_OK;
}

// column J of T for every process: t_J = (-beta T_J S_J^t s_J; beta)
static rhqr_status arnoldi_tcol(ArnoldiState &a, cudaStream_t st) {
  const int32_t J = a.j, M = a.M, B = a.nrhs;
  const int64_t p = (int64_t)a.view.k + M;
  dim3 g((unsigned)std::max(1, J), 2, (unsigned)B);
  RHQR_CUDA_TRY(launch_pdl(left_dots_kernel, g, dim3(256), 0, st, (const double *)a.S, a.lds, p, J, J,
                           (const double *)a.z, 0, a.d, a.v, 0, a.lds * M, p, (int64_t)M));
  RHQR_LAUNCH_CHECK();
  RHQR_CUDA_TRY(launch_pdl(left_tcol_coef_kernel, dim3((unsigned)B), dim3(1024), 0, st, a.T, M, J,
                           (const double *)a.beta, (const double *)a.d, (const double *)a.v, 0, a.c, 0,
                           (int64_t)M * M, (int64_t)M));
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

// refresh `w` (n x nrhs) with the reflectors 0..J-1 (coefficients in a.c),
// store it as column J of U, sketch it into a.y (fused), then take reflector J.
template <class T>
static rhqr_status arnoldi_reflect(ArnoldiState &a, const T *w, double *h, rhqr_info *info, cudaStream_t st) {
  const int32_t J = a.j, M = a.M, B = a.nrhs;
  const int64_t p = (int64_t)a.view.k + M;
  // the column kernel reads W[J * ldw + i]: present w as column J of a virtual matrix
  const T *Wbase = w - (int64_t)J * a.n;
  ColArgs ca{Wbase, a.n, a.U, a.ldu, a.n, M, J, a.c, a.gamma, a.y, a.scaling == 0 ? 1 : 0, 0, M,
             Batch{a.n, a.ldu * M, M, p, a.stage_elems}};
  const double scale = 1.0 / sqrt((double)a.view.k);
  if (a.view.kind == RHQR_SKETCH_SRHT) {
    RHQR_TRY(launch_refresh<T>(ca, (unsigned)B, st));
    RHQR_TRY(column_srht<T>(ca, a.view, (T *)a.stage, (unsigned)B, st));
    RHQR_CUDA_TRY(launch_pdl(left_srht_combine_kernel<T>, dim3((unsigned)ceil_div(a.view.k, 8), (unsigned)B),
                             dim3(256), 0, st, (const T *)a.stage, a.view.N1, a.view.d2, a.view.sample_i1,
                             a.view.sample_slot, a.view.k, M, scale, a.y, a.stage_elems, p));
    RHQR_LAUNCH_CHECK();
  } else {
    const dim3 gg((unsigned)ceil_div(a.n, LG_RB), (unsigned)B);
    switch (a.view.omega_dtype) {
      case RHQR_F64:
        left_column_gauss_kernel<T, double><<<gg, LG_RB, 0, st>>>(ca, (const double *)a.view.G, a.view.ldg, a.view.k,
                                                                  (double *)a.stage);
        break;
      case RHQR_F32:
        left_column_gauss_kernel<T, float><<<gg, LG_RB, 0, st>>>(ca, (const float *)a.view.G, a.view.ldg, a.view.k,
                                                                 (double *)a.stage);
        break;
      case RHQR_BF16:
        left_column_gauss_kernel<T, __nv_bfloat16><<<gg, LG_RB, 0, st>>>(
            ca, (const __nv_bfloat16 *)a.view.G, a.view.ldg, a.view.k, (double *)a.stage);
        break;
      default:
        left_column_gauss_kernel<T, __half><<<gg, LG_RB, 0, st>>>(ca, (const __half *)a.view.G, a.view.ldg, a.view.k,
                                                                  (double *)a.stage);
        break;
    }
    RHQR_LAUNCH_CHECK();
    left_gauss_reduce_kernel<<<dim3((unsigned)ceil_div(a.view.k, 128), (unsigned)B), 128, 0, st>>>(
        (const double *)a.stage, (int32_t)ceil_div(a.n, LG_RB), a.view.k, M, scale, a.y, a.stage_elems, p);
    RHQR_LAUNCH_CHECK();
  }
  // RHVector at column J; its "R column" is the Hessenberg column h (M entries per process)
  RhvBatch bb{p, a.lds * M, M, M, a.ldu * M, 4};
  RHQR_CUDA_TRY(launch_pdl(left_rhvector_kernel<T>, dim3((unsigned)B), dim3(256), 0, st, (const double *)a.y, p, M, J,
                           a.scaling, a.S, a.lds, h - (int64_t)J * M, a.beta, a.gamma, (T *)a.U, a.ldu, info, a.stop,
                           bb));
  RHQR_LAUNCH_CHECK();
  RHQR_TRY(arnoldi_tcol(a, st));
  a.j = J + 1;
  return RHQR_OK;
}

// q_J = e_J - U_{J+1} T_{J+1} S_{J+1}^t e_J  (J = the newest reflector)
template <class T>
static rhqr_status arnoldi_basis(ArnoldiState &a, T *q, cudaStream_t st) {
  const int32_t J = a.j - 1, B = a.nrhs;
  RHQR_CUDA_TRY(launch_pdl(arnoldi_coef_kernel, dim3((unsigned)B), dim3(1024), 0, st, (const double *)a.T, a.M,
                           (const double *)a.S, a.lds, J, (const double *)a.gamma, a.coef, a.lds * a.M));
  RHQR_LAUNCH_CHECK();
  // float32 basis: the vector kernel (its float64 form would stay bound by the
  // FP64 rate, so the float64 basis keeps the one-chain float64 sum)
  constexpr int V = Vec16<T>::V;
  const bool aligned = a.ldu % V == 0 && ((uintptr_t)a.U % 16) == 0 && ((uintptr_t)q % 16) == 0 &&
                       (B == 1 || a.n % V == 0);
  if (sizeof(T) == 4 && aligned) {
    const int64_t units = ceil_div(a.n, V);
    const dim3 g((unsigned)std::min<int64_t>(ceil_div(units, 256), std::max<int64_t>(1, 152 * 8 / (int64_t)B)),
                 (unsigned)B);
    RHQR_CUDA_TRY(launch_pdl(arnoldi_q_vec_kernel<T>, g, dim3(256), 0, st, (const T *)a.U, a.ldu, a.n, J,
                             (const double *)a.coef, q, a.ldu * a.M, a.M));
  } else {
    arnoldi_q_kernel<T><<<dim3((unsigned)ceil_div(a.n, 256), (unsigned)B), 256, 0, st>>>(
        (const T *)a.U, a.ldu, a.n, J, a.coef, q, a.ldu * a.M, a.M);
  }
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

template <class T>
static rhqr_status arnoldi_begin_t(ArnoldiState &a, const T *r0, double *h0, T *q1, rhqr_info *info,
                                   cudaStream_t st) {
  a.j = 0;
  RHQR_CUDA_TRY(cudaMemsetAsync(a.stop, 0, 4 * sizeof(int) * a.nrhs, st));
  RHQR_CUDA_TRY(cudaMemsetAsync(a.T, 0, sizeof(double) * a.M * a.M * a.nrhs, st));
  RHQR_TRY(arnoldi_reflect<T>(a, r0, h0, info, st));
  if (q1 != nullptr) RHQR_TRY(arnoldi_basis<T>(a, q1, st));
  return RHQR_OK;
}

template <class T>
static rhqr_status arnoldi_step_t(ArnoldiState &a, const T *w, double *h, T *qn, rhqr_info *info, cudaStream_t st) {
  const int32_t J = a.j, M = a.M, B = a.nrhs;
  const int64_t p = (int64_t)a.view.k + M;
  // z = Psi w (the sketches of A q_j of every process), then c = T_J^t S_J^t z
  RHQR_TRY(sketch_apply_simt(a.view, M, w, sizeof(T) == 8 ? RHQR_F64 : RHQR_F32, a.n, B, a.n, a.z, p, a.aws,
                             a.aws_bytes, st));
  dim3 g((unsigned)J, 2, (unsigned)B);
  RHQR_CUDA_TRY(launch_pdl(left_dots_kernel, g, dim3(256), 0, st, (const double *)a.S, a.lds, p, 0, 0,
                           (const double *)a.z, J, a.d, a.v, 0, a.lds * M, p, (int64_t)M));
  RHQR_LAUNCH_CHECK();
  RHQR_CUDA_TRY(launch_pdl(left_tcol_coef_kernel, dim3((unsigned)B), dim3(1024), 0, st, a.T, M, -1,
                           (const double *)a.beta, (const double *)a.d, (const double *)a.v, J, a.c, 0,
                           (int64_t)M * M, (int64_t)M));
  RHQR_LAUNCH_CHECK();
  RHQR_TRY(arnoldi_reflect<T>(a, w, h, info, st));
  if (qn != nullptr) RHQR_TRY(arnoldi_basis<T>(a, qn, st));
  return RHQR_OK;
}

// the newest column of U is stored unscaled (deferred scaling): scale it in a copy
rhqr_status arnoldi_scale_copy(const ArnoldiState &a, void *Udst, int64_t ldu, cudaStream_t st) {
  if (a.j < 1) return RHQR_OK;
  const dim3 g((unsigned)ceil_div(a.n, 256), (unsigned)a.nrhs);
  if (a.dtype == RHQR_F64)
    left_scale_last_kernel<double><<<g, 256, 0, st>>>((double *)Udst, ldu, a.n, a.j - 1, a.gamma, a.scaling == 0,
                                                      ldu * a.M, a.M);
  else
    left_scale_last_kernel<float><<<g, 256, 0, st>>>((float *)Udst, ldu, a.n, a.j - 1, a.gamma, a.scaling == 0,
                                                     ldu * a.M, a.M);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

rhqr_status arnoldi_begin(ArnoldiState &a, const void *r0, double *h0, void *q1, rhqr_info *info, cudaStream_t st) {
  if (a.dtype == RHQR_F64) return arnoldi_begin_t<double>(a, (const double *)r0, h0, (double *)q1, info, st);
  return arnoldi_begin_t<float>(a, (const float *)r0, h0, (float *)q1, info, st);
}

rhqr_status arnoldi_step(ArnoldiState &a, const void *w, double *h, void *qn, rhqr_info *info, cudaStream_t st) {
  if (a.dtype == RHQR_F64) return arnoldi_step_t<double>(a, (const double *)w, h, (double *)qn, info, st);
  return arnoldi_step_t<float>(a, (const float *)w, h, (float *)qn, info, st);
}

// ---------------------------------------------------------------------------
// RHQR-GMRES (Algorithm 8): the sketched minimal-residual solution
// ---------------------------------------------------------------------------

// y = argmin || h0 - H y || for the (m+1) x m Hessenberg H (eq. rgmresopti),
// by Givens rotations in float64: thread 0 rotates column after column (the
// column being rotated and the rotations live in shared memory, the triangle
// R goes to `Rs`, ld = m), then the warp back-substitutes by columns (lane i
// keeps the partial sum of row i).  res = || h0 - H y ||.  One warp per
// process (blockIdx.x): H at H + b bs_H, h0 at h0 + b M, y at y + b bs_y.
__global__ void arnoldi_lsq_kernel(const double *H, int64_t ldh, int32_t m, int32_t M, const double *h0, double *Rs,
                                   double *y, double *res, int64_t bs_H, int64_t bs_y) {
  extern __shared__ double sh[];
  {
    const int64_t b = blockIdx.x;
    H += b * bs_H;
    h0 += b * M;
    Rs += b * (int64_t)M * M;
    y += b * bs_y;
    res += b;
  }
  double *col = sh;          // [m + 1]
  double *cs = sh + m + 1;   // [m]
  double *sn = cs + m;       // [m]
  double *g = sn + m;        // [m + 1]
  const int lane = threadIdx.x;
  for (int i = lane; i <= m; i += 32) g[i] = h0[i];
  __syncwarp();
  if (lane == 0) {
    for (int j = 0; j < m; ++j) {
      for (int i = 0; i <= j + 1; ++i) col[i] = H[(int64_t)j * ldh + i];
      for (int i = 0; i < j; ++i) {
        const double a = col[i], b = col[i + 1];
        col[i] = cs[i] * a + sn[i] * b;
        col[i + 1] = cs[i] * b - sn[i] * a;
      }
      const double a = col[j], b = col[j + 1];
      const double d = hypot(a, b);
      const double c = d == 0.0 ? 1.0 : a / d, sv = d == 0.0 ? 0.0 : b / d;
      cs[j] = c;
      sn[j] = sv;
      col[j] = d;
      const double g0 = g[j], g1 = g[j + 1];
      g[j] = c * g0 + sv * g1;
      g[j + 1] = c * g1 - sv * g0;
      for (int i = 0; i <= j; ++i) Rs[(int64_t)j * m + i] = col[i];
    }
    // entries of h0 below row m are not reached by H's first m columns
    double tail = g[m] * g[m];
    for (int i = m + 1; i < M; ++i) tail += h0[i] * h0[i];
    *res = sqrt(tail);
  }
  __syncwarp();
  __threadfence_block();
  // back substitution R y = g[0:m], by columns: y_l = s_l / R_ll, then s_i -= R_il y_l
  double sacc[32];
#pragma unroll
  for (int t = 0; t < 32; ++t) sacc[t] = 0.0;
  for (int l = m - 1; l >= 0; --l) {
    const int owner = l & 31, slot = l >> 5;
    double yl = 0.0;
    if (lane == owner) {
      double sv = 0.0;
#pragma unroll
      for (int t = 0; t < 32; ++t)
        if (t == slot) sv = sacc[t];
      yl = (g[l] - sv) / Rs[(int64_t)l * m + l];
      y[l] = yl;
    }
    yl = __shfl_sync(0xffffffffu, yl, owner);
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      const int i = lane + 32 * t;
      if (i < l) sacc[t] += Rs[(int64_t)l * m + i] * yl;
    }
  }
}

// coef = T_m (S_m^t y) with S_m = rows 0..m-1 of S's first m columns (the
// identity top block of Psi keeps [y; 0] unchanged): v_i = sum_{j >= i} S_ji y_j,
// coef_l = sum_{i >= l} T_li v_i.  One block per process.
__global__ void arnoldi_solution_coef_kernel(const double *T, int32_t M, const double *S, int64_t lds, int32_t m,
                                             const double *y, double *v, double *coef, int64_t bs_S, int64_t bs_y) {
  {
    const int64_t b = blockIdx.x;
    T += b * (int64_t)M * M;
    S += b * bs_S;
    y += b * bs_y;
    v += b * M;
    coef += b * M;
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double acc = 0.0;
    for (int j = i; j < m; ++j) acc += S[(int64_t)i * lds + j] * y[j];
    v[i] = acc;
  }
  __syncthreads();
  for (int l = threadIdx.x; l < m; l += blockDim.x) {
    double acc = 0.0;
    for (int i = l; i < m; ++i) acc += T[(int64_t)i * M + l] * v[i];
    coef[l] = acc;
  }
}

// x = x0 + [y; 0] - U_m coef (columns 0..m-1 of U are scaled once m steps were
// taken); process blockIdx.y, its x0 and x at + b n.
template <class T, class TX>
__global__ void arnoldi_x_kernel(const T *U, int64_t ldu, int64_t n, int32_t m, const double *coef,
                                 const double *y, const TX *x0, TX *x, int64_t bs_U, int32_t M, int64_t bs_y) {
  {
    const int64_t b = blockIdx.y;
    U += b * bs_U;
    coef += b * M;
    y += b * bs_y;
    x0 += b * n;
    x += b * n;
  }
  __shared__ double c_s[1024];
  for (int l = threadIdx.x; l < m; l += blockDim.x) c_s[l] = coef[l];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = (double)x0[i] + (i < m ? y[i] : 0.0);
  for (int l = 0; l < m; ++l) acc -= (double)U[(int64_t)l * ldu + i] * c_s[l];
  x[i] = (TX)acc;
}

size_t arnoldi_solution_scratch_doubles(int32_t M, int32_t nrhs) {
  return ((size_t)M * M + 2 * (size_t)M) * (size_t)nrhs;
}

rhqr_status arnoldi_solution(const ArnoldiState &a, double *scratch, const double *H, int64_t ldh, int32_t m,
                             const double *h0, const void *x0, void *x, int32_t xdt, double *y, double *res,
                             cudaStream_t st) {
  if (m < 1 || m > a.j - 1 || m > a.M - 1 || ldh < m + 1) return RHQR_EINVAL;
  if (xdt != RHQR_F64 && xdt != RHQR_F32) return RHQR_EINVAL;
  const int32_t B = a.nrhs, M = a.M;
  double *Rs = scratch, *v = scratch + (size_t)M * M * B, *coef = v + (size_t)M * B;
  const int64_t bs_H = ldh * (M - 1), bs_y = M - 1;  // per process: H is (mmax+1) x mmax, y has mmax entries
  const size_t smem = sizeof(double) * (4 * (size_t)m + 2);  // column, cosines, sines, rotated h0
  arnoldi_lsq_kernel<<<(unsigned)B, 32, smem, st>>>(H, ldh, m, M, h0, Rs, y, res, bs_H, bs_y);
  RHQR_LAUNCH_CHECK();
  if (x == nullptr) return RHQR_OK;
  arnoldi_solution_coef_kernel<<<(unsigned)B, 256, 0, st>>>(a.T, M, a.S, a.lds, m, y, v, coef, a.lds * M, bs_y);
  RHQR_LAUNCH_CHECK();
  const dim3 grid((unsigned)ceil_div(a.n, (int64_t)256), (unsigned)B);
  if (a.dtype == RHQR_F64 && xdt == RHQR_F64)
    arnoldi_x_kernel<double, double><<<grid, 256, 0, st>>>((const double *)a.U, a.ldu, a.n, m, coef, y,
                                                           (const double *)x0, (double *)x, a.ldu * M, M, bs_y);
  else if (a.dtype == RHQR_F64)
    arnoldi_x_kernel<double, float><<<grid, 256, 0, st>>>((const double *)a.U, a.ldu, a.n, m, coef, y,
                                                          (const float *)x0, (float *)x, a.ldu * M, M, bs_y);
  else if (xdt == RHQR_F64)
    arnoldi_x_kernel<float, double><<<grid, 256, 0, st>>>((const float *)a.U, a.ldu, a.n, m, coef, y,
                                                          (const double *)x0, (double *)x, a.ldu * M, M, bs_y);
  else
    arnoldi_x_kernel<float, float><<<grid, 256, 0, st>>>((const float *)a.U, a.ldu, a.n, m, coef, y,
                                                         (const float *)x0, (float *)x, a.ldu * M, M, bs_y);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

}  // namespace rhqr
