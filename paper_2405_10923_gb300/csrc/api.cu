// C ABI of the library (include/rhqr.h): argument checks, sketch handles,
// workspace carving and the sequencing of the kernels of each entry point.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "apply.cuh"
#include "common.cuh"
#include "left.cuh"
#include "rng.cuh"
#include "sketch.cuh"
#include "sketch_tc.cuh"
#include "small.cuh"
#include "solve_tc.cuh"
#include "solve_inv_tc.cuh"

struct rhqr_sketch_s {
  rhqr::SketchView view;
  uint64_t seed;
  void *mem;  // one device allocation for everything below
  size_t mem_bytes;
};

struct rhqr_arnoldi_s {
  rhqr::ArnoldiState st;
  void *mem;
  double *lsq;  // scratch of rhqr_arnoldi_solution (the Givens triangle, coefficients)
};

namespace rhqr {

const SketchView *sketch_view_of(rhqr_sketch s) { return &s->view; }

static bool valid_dtype_hd(int32_t t) { return t == RHQR_F64 || t == RHQR_F32; }
static bool valid_dtype_any(int32_t t) { return t >= RHQR_F64 && t <= RHQR_F16; }

// Kronecker split of the SRHT transform: N = N1 * N2 with N2 <= 8192 (8192
// float64 fit in 64 KiB of shared memory).
static int32_t srht_n2(int64_t N) { return (int32_t)std::min<int64_t>(N, 8192); }

}  // namespace rhqr

using namespace rhqr;

extern "C" {

const char *rhqr_status_string(rhqr_status s) {
  switch (s) {
    case RHQR_OK: return "ok";
    case RHQR_EINVAL: return "invalid argument";
    case RHQR_ENOMEM: return "out of memory or workspace too small";
    case RHQR_ECUDA: return "CUDA runtime error";
    case RHQR_EBREAKDOWN: return "breakdown: column lies in the kernel of the sketch";
    case RHQR_ENONFINITE: return "non-finite value";
    case RHQR_ETIMEOUT: return "device-side wait timed out";
    case RHQR_ENOTSUP: return "not supported";
  }
  return "unknown status";
}

int32_t rhqr_version(void) { return 1; }
int32_t rhqr_built_arch(void) { return 103; }

void rhqr_default_opts(rhqr_opts *o) {
  if (o == nullptr) return;
  std::memset(o, 0, sizeof(*o));
  o->alg = RHQR_ALG_REC;
  o->passes = 1;
  o->limbs_first = 2;
  o->limbs_refine = 2;
  o->want_U = 0;
  o->want_Q = 1;
  o->scaling = 0;
  o->wait_budget = 0;
  o->block_size = 32;
  o->column_scaling = 0;
}

rhqr_status rhqr_sketch_create(int64_t n, int32_t k, int32_t kind, uint64_t seed, int32_t omega_dtype,
                               rhqr_stream_t stream, rhqr_sketch *out) {
  if (out == nullptr) return RHQR_EINVAL;
  *out = nullptr;
  if (n < 2 || k < 1) return RHQR_EINVAL;
  if (kind != RHQR_SKETCH_GAUSSIAN && kind != RHQR_SKETCH_SRHT) return RHQR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  rhqr_sketch s = new (std::nothrow) rhqr_sketch_s();
  if (s == nullptr) return RHQR_ENOMEM;
  SketchView &v = s->view;
  std::memset(&v, 0, sizeof(v));
  v.n = n;
  v.k = k;
  v.kind = kind;
  s->seed = seed;
  if (kind == RHQR_SKETCH_SRHT) {
    int64_t N = 1;
    while (N < n) N <<= 1;
    if (k > N || N > (int64_t(1) << 30)) {
      delete s;
      return RHQR_EINVAL;
    }
    v.N = N;
    v.N2 = srht_n2(N);
    v.N1 = (int32_t)(N / v.N2);
    v.omega_dtype = RHQR_F64;
    int64_t words = ceil_div(N, 32);
    int64_t nb = ceil_div(N, 1024);
    Carver c(nullptr, 0);
    c.take<uint32_t>(words);
    c.take<int32_t>(k);       // rows
    c.take<int32_t>(k);       // i2_list (<= k distinct)
    c.take<int32_t>(k);       // sample_i1
    c.take<int32_t>(k);       // sample_slot
    c.take<char>(2048 + 4 * nb);  // selection scratch
    s->mem_bytes = c.used() + 256;
    if (cudaMalloc(&s->mem, s->mem_bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      delete s;
      return RHQR_ENOMEM;
    }
    Carver d(s->mem, s->mem_bytes);
    uint32_t *bits = d.take<uint32_t>(words);
    int32_t *rows = d.take<int32_t>(k);
    int32_t *i2 = d.take<int32_t>(k);
    int32_t *si1 = d.take<int32_t>(k);
    int32_t *sslot = d.take<int32_t>(k);
    char *scratch = d.take<char>(2048 + 4 * nb);
    rhqr_status r = make_srht_operator(N, k, seed, bits, rows, scratch, 2048 + 4 * nb, st);
    if (r != RHQR_OK) {
      cudaFree(s->mem);
      delete s;
      return r;
    }
    // Kronecker bookkeeping of the sampled rows (host, k integers)
    std::vector<int32_t> hrows(k), hi2, hi1(k), hslot(k);
    if (cudaMemcpy(hrows.data(), rows, sizeof(int32_t) * k, cudaMemcpyDeviceToHost) != cudaSuccess) {
      (void)cudaGetLastError();
      cudaFree(s->mem);
      delete s;
      return RHQR_ECUDA;
    }
    for (int r2 = 0; r2 < k; ++r2) hi2.push_back(hrows[r2] % v.N2);
    std::sort(hi2.begin(), hi2.end());
    hi2.erase(std::unique(hi2.begin(), hi2.end()), hi2.end());
    for (int r2 = 0; r2 < k; ++r2) {
      hi1[r2] = hrows[r2] / v.N2;
      hslot[r2] = (int32_t)(std::lower_bound(hi2.begin(), hi2.end(), hrows[r2] % v.N2) - hi2.begin());
    }
    v.d2 = (int32_t)hi2.size();
    cudaMemcpy(i2, hi2.data(), sizeof(int32_t) * v.d2, cudaMemcpyHostToDevice);
    cudaMemcpy(si1, hi1.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice);
    if (cudaMemcpy(sslot, hslot.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice) != cudaSuccess) {
      (void)cudaGetLastError();
      cudaFree(s->mem);
      delete s;
      return RHQR_ECUDA;
    }
    v.sign_bits = bits;
    v.rows = rows;
    v.i2_list = i2;
    v.sample_i1 = si1;
    v.sample_slot = sslot;
  } else {
    if (!valid_dtype_any(omega_dtype)) {
      delete s;
      return RHQR_EINVAL;
    }
    v.N = n;
    v.omega_dtype = omega_dtype;
    size_t es = dtype_size(omega_dtype);
    // rows padded to 16 bytes (TMA-compatible strides)
    int64_t ldg = (int64_t)align_up((size_t)n * es, 16) / (int64_t)es;
    v.ldg = ldg;
    // 16-bit operators feed the tensor-core sketch, which reads them in tile order
    const bool tiles = omega_dtype == RHQR_BF16 || omega_dtype == RHQR_F16;
    Carver c(nullptr, 0);
    c.take<char>((size_t)k * ldg * es);
    c.take<double>(32);
    if (tiles) c.take<char>(operator_tiles_bytes(n, k));
    s->mem_bytes = c.used() + 256;
    if (cudaMalloc(&s->mem, s->mem_bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      delete s;
      return RHQR_ENOMEM;
    }
    Carver d(s->mem, s->mem_bytes);
    char *gmem = d.take<char>((size_t)k * ldg * es);
    double *coef = d.take<double>(32);
    char *gt = tiles ? d.take<char>(operator_tiles_bytes(n, k)) : nullptr;
    v.G = gmem;
    v.Gt = gt;
    v.gt_nkb = tiles ? operator_tiles_nkb(n) : 0;
    if (ldg != n) RHQR_CUDA_TRY(cudaMemsetAsync(gmem, 0, (size_t)k * ldg * es, st));
    rhqr_status r = make_gaussian_operator(n, k, seed, omega_dtype, gmem, ldg, coef, st);
    if (r == RHQR_OK && tiles) r = make_operator_tiles(gmem, ldg, n, k, gt, st);
    if (r != RHQR_OK) {
      cudaFree(s->mem);
      delete s;
      return r;
    }
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    (void)cudaGetLastError();
    cudaFree(s->mem);
    delete s;
    return RHQR_ECUDA;
  }
  *out = s;
  return RHQR_OK;
}

rhqr_status rhqr_sketch_destroy(rhqr_sketch s) {
  if (s == nullptr) return RHQR_OK;
  cudaError_t e = cudaFree(s->mem);
  delete s;
  return e == cudaSuccess ? RHQR_OK : RHQR_ECUDA;
}

rhqr_status rhqr_sketch_shape(rhqr_sketch s, int64_t *n, int32_t *k, int32_t *kind, int64_t *N,
                              int32_t *omega_dtype) {
  if (s == nullptr) return RHQR_EINVAL;
  if (n) *n = s->view.n;
  if (k) *k = s->view.k;
  if (kind) *kind = s->view.kind;
  if (N) *N = s->view.N;
  if (omega_dtype) *omega_dtype = s->view.omega_dtype;
  return RHQR_OK;
}

rhqr_status rhqr_sketch_export(rhqr_sketch s, int8_t *signs, int32_t *rows, void *G, int64_t ldg,
                               rhqr_stream_t stream) {
  if (s == nullptr) return RHQR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const SketchView &v = s->view;
  if (v.kind == RHQR_SKETCH_SRHT) {
    if (signs) RHQR_TRY(export_signs(v.sign_bits, signs, v.N, st));
    if (rows) RHQR_CUDA_TRY(cudaMemcpyAsync(rows, v.rows, sizeof(int32_t) * v.k, cudaMemcpyDeviceToDevice, st));
  } else if (G != nullptr) {
    if (ldg < v.n) return RHQR_EINVAL;
    size_t es = dtype_size(v.omega_dtype);
    RHQR_CUDA_TRY(cudaMemcpy2DAsync(G, ldg * es, v.G, v.ldg * es, v.n * es, v.k, cudaMemcpyDeviceToDevice, st));
  }
  return RHQR_OK;
}

rhqr_status rhqr_sketch_apply_workspace(rhqr_sketch s, int32_t m, int32_t xt, int64_t n, int32_t c,
                                        size_t *bytes) {
  if (s == nullptr || bytes == nullptr || !valid_dtype_hd(xt) || c < 1 || m < 0 || n <= m) return RHQR_EINVAL;
  *bytes = sketch_apply_workspace_bytes(s->view, m, xt, n, c);
  if (xt == RHQR_F32 && sketch_tc_supported(s->view, n, m, c))
    *bytes = std::max(*bytes, sketch_tc_workspace_bytes(s->view, n, m, c));
  return RHQR_OK;
}

static rhqr_status check_sketch_shape(const SketchView &v, int64_t n, int32_t m) {
  if (m < 0 || n <= m || m > v.k) return RHQR_EINVAL;
  if (v.kind == RHQR_SKETCH_GAUSSIAN && n != v.n) return RHQR_EINVAL;
  if (v.kind == RHQR_SKETCH_SRHT && n > v.N) return RHQR_EINVAL;
  return RHQR_OK;
}

rhqr_status rhqr_sketch_apply(rhqr_sketch s, int32_t m, const void *X, int32_t xt, int64_t n, int32_t c,
                              int64_t ldx, double *Z, int64_t ldz, void *ws, size_t ws_bytes,
                              rhqr_stream_t stream) {
  if (s == nullptr || X == nullptr || Z == nullptr || !valid_dtype_hd(xt) || c < 1) return RHQR_EINVAL;
  RHQR_TRY(check_sketch_shape(s->view, n, m));
  if (ldx < n || ldz < (int64_t)s->view.k + m) return RHQR_EINVAL;
  // float32 data with a 16-bit Gaussian operator: tensor cores, exact 3-limb split
  if (xt == RHQR_F32 && sketch_tc_supported(s->view, n, m, c) && ldx % 4 == 0 && ((uintptr_t)X % 16) == 0)
    return sketch_apply_tc(s->view, m, (const float *)X, n, c, ldx, 3, Z, ldz, ws, ws_bytes, nullptr, 0,
                           (cudaStream_t)stream);
  return sketch_apply_simt(s->view, m, X, xt, n, c, ldx, Z, ldz, ws, ws_bytes, (cudaStream_t)stream);
}

static rhqr_status check_rows(const SketchView &v, int32_t m, int32_t xt, int64_t row0, int64_t rows, int32_t c) {
  if (!valid_dtype_hd(xt) || c < 1 || rows < 1 || row0 < 0 || m < 0 || m > v.k || m >= v.n) return RHQR_EINVAL;
  if (row0 + rows > v.n) return RHQR_EINVAL;
  if (v.kind == RHQR_SKETCH_SRHT && row0 % v.N2 != 0) return RHQR_EINVAL;  // shards start on a segment
  return RHQR_OK;
}

rhqr_status rhqr_sketch_apply_rows_workspace(rhqr_sketch s, int32_t m, int32_t xt, int64_t row0, int64_t rows,
                                             int32_t c, size_t *bytes) {
  if (s == nullptr || bytes == nullptr) return RHQR_EINVAL;
  RHQR_TRY(check_rows(s->view, m, xt, row0, rows, c));
  *bytes = sketch_rows_workspace_bytes(s->view, m, xt, row0, rows, c);
  return RHQR_OK;
}

rhqr_status rhqr_sketch_apply_rows(rhqr_sketch s, int32_t m, const void *X, int32_t xt, int64_t row0, int64_t rows,
                                   int32_t c, int64_t ldx, double *Z, int64_t ldz, void *ws, size_t ws_bytes,
                                   rhqr_stream_t stream) {
  if (s == nullptr || X == nullptr || Z == nullptr) return RHQR_EINVAL;
  RHQR_TRY(check_rows(s->view, m, xt, row0, rows, c));
  if (ldx < rows || ldz < (int64_t)s->view.k + m) return RHQR_EINVAL;
  if (ws == nullptr || ws_bytes < sketch_rows_workspace_bytes(s->view, m, xt, row0, rows, c)) return RHQR_ENOMEM;
  return sketch_apply_rows_simt(s->view, m, X, xt, row0, rows, c, ldx, Z, ldz, ws, ws_bytes, (cudaStream_t)stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// recRHQR orchestration
// ---------------------------------------------------------------------------

struct RecBuffers {
  double *Z, *Spass, *Rpass, *Racc, *Rtmp, *beta, *SS, *StZ, *M, *Gm;
  char *TriT, *GT;
  float *TriT64;  // padded to a multiple of the tensor-core panel width
  double *Rinv;   // R^{-1} of the pass (tensor-core product solve)
  double *colnorm;  // column norms of the pass's sketch (column_scaling)
  char *hqr_ws;
  size_t hqr_bytes;
  char *sk_ws;
  size_t sk_bytes;
};

static size_t sketch_ws_for_factor(const SketchView &v, int64_t n, int32_t m, int32_t wt, const rhqr_opts &o) {
  size_t b = sketch_apply_workspace_bytes(v, m, wt, n, m);
  if (v.kind == RHQR_SKETCH_GAUSSIAN && (v.omega_dtype == RHQR_BF16 || v.omega_dtype == RHQR_F16) &&
      wt == RHQR_F32)
    b = std::max(b, sketch_tc_workspace_bytes(v, n, m, m));
  (void)o;
  return b;
}

static rhqr_status carve_rec(Carver &c, const SketchView &v, int64_t n, int32_t m, int32_t wt, const rhqr_opts &o,
                             RecBuffers &b) {
  int64_t p = (int64_t)v.k + m;
  b.Z = c.take<double>((size_t)p * m);
  b.Spass = c.take<double>((size_t)p * m);
  b.Rpass = c.take<double>((size_t)m * m);
  b.Racc = c.take<double>((size_t)m * m);
  b.Rtmp = c.take<double>((size_t)m * m);
  b.beta = c.take<double>(m);
  b.SS = c.take<double>((size_t)m * m);
  b.StZ = c.take<double>((size_t)m * m);
  b.M = c.take<double>((size_t)m * m);
  b.Gm = c.take<double>((size_t)m * m);
  b.TriT = c.take<char>(small_padded_bytes(m));
  b.GT = c.take<char>(small_padded_bytes(m));
  {
    int64_t mp64 = ceil_div(m, kSolvePanel) * kSolvePanel;
    b.TriT64 = c.take<float>((size_t)mp64 * mp64);
    b.Rinv = c.take<double>((size_t)m * m);
    b.colnorm = c.take<double>(m);
  }
  b.hqr_bytes = hqr_workspace_bytes(p, m);
  b.hqr_ws = c.take<char>(b.hqr_bytes);
  b.sk_bytes = sketch_ws_for_factor(v, n, m, wt, o);
  b.sk_ws = c.take<char>(b.sk_bytes);
  return c.overflow() ? RHQR_ENOMEM : RHQR_OK;
}

static rhqr_status sketch_for_pass(const SketchView &v, int32_t m, const void *X, int32_t wt, int64_t n,
                                   int64_t ldx, double *Z, int64_t ldz, int limbs, RecBuffers &b, rhqr_info *info,
                                   long long budget, cudaStream_t st) {
  if (v.kind == RHQR_SKETCH_GAUSSIAN && (v.omega_dtype == RHQR_BF16 || v.omega_dtype == RHQR_F16) &&
      wt == RHQR_F32 && sketch_tc_supported(v, n, m, m)) {
    return sketch_apply_tc(v, m, (const float *)X, n, m, ldx, limbs, Z, ldz, b.sk_ws, b.sk_bytes, info, budget, st);
  }
  return sketch_apply_simt(v, m, X, wt, n, m, ldx, Z, ldz, b.sk_ws, b.sk_bytes, st);
}

// Q = X Tri^{-1} over all n rows.  float32 data with m <= 256 runs on the
// tensor cores: by default as the product with the explicit inverse (limb
// products chosen for float32-level results), with opts.solve = 1 as the
// row-wise substitution; other cases use the SIMT substitution.
template <class T>
static rhqr_status solve_rows(const T *X, int64_t ldx, int64_t n, int32_t m, const double *Tri, T *Q, int64_t ldq,
                              RecBuffers &b, const rhqr_opts &o, rhqr_info *info, long long budget, cudaStream_t st);
template <>
rhqr_status solve_rows<float>(const float *X, int64_t ldx, int64_t n, int32_t m, const double *Tri, float *Q,
                              int64_t ldq, RecBuffers &b, const rhqr_opts &o, rhqr_info *info, long long budget,
                              cudaStream_t st) {
  if (o.solve == 0 && solve_inv_tc_supported(m) && (X != Q || ldx == ldq)) {
    RHQR_TRY(upper_inverse(Tri, m, b.Rinv, st));
    return rows_solve_inv_tc(X, ldx, n, m, b.Rinv, 0, Q, ldq, info, budget, st);
  }
  if (solve_tc_supported(m)) {
    int32_t mp64 = (int32_t)(ceil_div(m, kSolvePanel) * kSolvePanel);
    RHQR_TRY(pad_transpose_to<float>(Tri, m, mp64, 1, b.TriT64, st));
    return rows_solve_tc(X, ldx, 0, n, m, b.TriT64, mp64, Q, ldq, info, budget, st);
  }
  RHQR_TRY(pad_transpose<float>(Tri, m, 1, (float *)b.TriT, st));
  return rows_solve<float>(X, ldx, 0, n, m, (const float *)b.TriT, Q, ldq, st);
}
template <>
rhqr_status solve_rows<double>(const double *X, int64_t ldx, int64_t n, int32_t m, const double *Tri, double *Q,
                               int64_t ldq, RecBuffers &b, const rhqr_opts &o, rhqr_info *info, long long budget,
                               cudaStream_t st) {
  (void)o, (void)info, (void)budget;
  RHQR_TRY(pad_transpose<double>(Tri, m, 1, (double *)b.TriT, st));
  return rows_solve<double>(X, ldx, 0, n, m, (const double *)b.TriT, Q, ldq, st);
}

template <class T>
static rhqr_status rec_typed(const SketchView &v, const T *W, int32_t wt, int64_t n, int32_t m, int64_t ldw,
                             const rhqr_opts &o, T *U, int64_t ldu, double *S, int64_t lds, double *Tm, double *R,
                             T *Q, int64_t ldq, RecBuffers &b, rhqr_info *info, cudaStream_t st) {
  const int64_t p = (int64_t)v.k + m;
  const long long budget = o.wait_budget > 0 ? o.wait_budget : kDefaultWaitBudget;
  const T *X = W;
  int64_t ldx = ldw;
  for (int pass = 0; pass < o.passes; ++pass) {
    const bool last = (pass == o.passes - 1);
    int limbs = pass == 0 ? o.limbs_first : o.limbs_refine;
    {
      PhaseScope ps(PH_SKETCH, st);
      RHQR_TRY(sketch_for_pass(v, m, X, wt, n, ldx, b.Z, p, limbs, b, info, budget, st));
    }
    double *Sdst = last ? S : b.Spass;
    int64_t ldsd = last ? lds : p;
    {
      PhaseScope ps(PH_HQR, st);
      // column equilibration: Householder QR of Z D^{-1} has the same reflectors
      // and R D^{-1}, so R = R~ D
      if (o.column_scaling) RHQR_TRY(equilibrate_columns(b.Z, p, p, m, b.colnorm, st));
      RHQR_TRY(householder_qr_small(b.Z, p, p, m, Sdst, ldsd, b.Rpass, b.beta, o.scaling, b.hqr_ws, b.hqr_bytes,
                                    info, budget, st));
      if (o.column_scaling) {
        RHQR_TRY(scale_columns(b.Rpass, m, m, m, b.colnorm, st));
        RHQR_TRY(scale_columns(b.Z, p, p, m, b.colnorm, st));  // Z again for M = ut(T^t S^t Z)
      }
    }
    if (pass == 0) {
      RHQR_TRY(copy_f64(b.Rpass, (int64_t)m * m, b.Racc, st));
    } else {
      RHQR_TRY(triu_mul(b.Rpass, b.Racc, m, b.Rtmp, st));
      RHQR_TRY(copy_f64(b.Rtmp, (int64_t)m * m, b.Racc, st));
    }
    if (last) {
      {
        PhaseScope ps(PH_TFACTOR, st);
        RHQR_TRY(t_factor_small(S, lds, p, m, b.beta, b.SS, Tm, st));
      }
      PhaseScope ps(PH_SOLVE, st);
      if (o.want_U) {
        // Algorithm 6: U_1 = S_{1:m}, U_2 solves X_2 = U_2 ut(T^t S^t Z); Q = [I;0] - U T U_1^t
        RHQR_TRY(m_factor(Tm, S, lds, b.Z, p, p, m, b.StZ, b.M, st));
        RHQR_TRY(t_u1t(Tm, S, lds, m, b.Gm, st));
        RHQR_TRY(pad_transpose<T>(b.M, m, 1, (T *)b.TriT, st));
        RHQR_TRY(pad_transpose<T>(b.Gm, m, 1, (T *)b.GT, st));
        RHQR_TRY(rows_solve_mul<T>(X, ldx, m, n - m, m, (const T *)b.TriT, (const T *)b.GT, U, ldu, Q, ldq, st));
        RHQR_TRY(top_from_s<T>(S, lds, m, U, ldu, st));
        if (Q != nullptr) RHQR_TRY(rows_form_q<T>(U, ldu, 0, m, m, (const T *)b.GT, Q, ldq, st));
      } else if (Q != nullptr) {
        RHQR_TRY(solve_rows<T>(X, ldx, n, m, b.Rpass, Q, ldq, b, o, info, budget, st));
      }
    } else {
      // Q_i = X_{i-1} R_i^{-1} becomes the next pass's input (in place in Q)
      PhaseScope ps(PH_SOLVE, st);
      RHQR_TRY(solve_rows<T>(X, ldx, n, m, b.Rpass, Q, ldq, b, o, info, budget, st));
      X = Q;
      ldx = ldq;
    }
  }
  RHQR_TRY(copy_f64(b.Racc, (int64_t)m * m, R, st));
  RHQR_TRY(info_passes(info, o.passes, st));
  return RHQR_OK;
}

extern "C" {

rhqr_status rhqr_workspace_size(rhqr_sketch s, int64_t n, int32_t m, int32_t wt, const rhqr_opts *opts,
                                size_t *bytes) {
  if (s == nullptr || bytes == nullptr || !valid_dtype_hd(wt) || m < 1) return RHQR_EINVAL;
  RHQR_TRY(check_sketch_shape(s->view, n, m));
  rhqr_opts o;
  if (opts) o = *opts;
  else rhqr_default_opts(&o);
  if (o.alg == RHQR_ALG_LEFT) {
    *bytes = left_workspace_bytes(s->view, n, m, wt);
    return RHQR_OK;
  }
  if (o.alg == RHQR_ALG_BLOCK) {
    *bytes = block_workspace_bytes(s->view, n, m, o.block_size, wt);
    return RHQR_OK;
  }
  Carver c(nullptr, 0);
  RecBuffers b;
  carve_rec(c, s->view, n, m, wt, o, b);
  *bytes = c.used() + 1024;
  return RHQR_OK;
}

rhqr_status rhqr_factor(rhqr_sketch s, const void *W, int32_t wt, int64_t n, int32_t m, int64_t ldw,
                        const rhqr_opts *opts, void *U, int64_t ldu, double *S, int64_t lds, double *T, double *R,
                        void *Q, int64_t ldq, void *ws, size_t ws_bytes, rhqr_info *info, rhqr_stream_t stream) {
  if (s == nullptr || W == nullptr || S == nullptr || T == nullptr || R == nullptr || info == nullptr)
    return RHQR_EINVAL;
  if (!valid_dtype_hd(wt) || m < 1) return RHQR_EINVAL;
  RHQR_TRY(check_sketch_shape(s->view, n, m));
  rhqr_opts o;
  if (opts) o = *opts;
  else rhqr_default_opts(&o);
  const int64_t p = (int64_t)s->view.k + m;
  if (ldw < n || lds < p) return RHQR_EINVAL;
  if ((o.scaling != 0 && o.scaling != 1) || (o.solve != 0 && o.solve != 1)) return RHQR_EINVAL;
  if (o.alg != RHQR_ALG_LEFT && o.alg != RHQR_ALG_REC && o.alg != RHQR_ALG_BLOCK) return RHQR_EINVAL;
  if (o.alg == RHQR_ALG_BLOCK && (o.block_size < 1 || o.block_size > 64)) return RHQR_EINVAL;
  if (o.column_scaling != 0 && o.column_scaling != 1) return RHQR_EINVAL;
  if (o.want_Q && (Q == nullptr || ldq < n)) return RHQR_EINVAL;
  if ((o.want_U || o.alg != RHQR_ALG_REC) && (U == nullptr || ldu < n)) return RHQR_EINVAL;
  if (o.alg == RHQR_ALG_REC && (o.passes < 1 || o.passes > 16)) return RHQR_EINVAL;
  if (o.alg == RHQR_ALG_REC && o.passes > 1 && !o.want_Q) return RHQR_EINVAL;  // Q holds the passes' iterates
  if (o.limbs_first < 1 || o.limbs_first > 3 || o.limbs_refine < 1 || o.limbs_refine > 3) return RHQR_EINVAL;
  if (m > 1024) return RHQR_ENOTSUP;
  cudaStream_t st = (cudaStream_t)stream;
  size_t need = 0;
  RHQR_TRY(rhqr_workspace_size(s, n, m, wt, &o, &need));
  if (ws == nullptr || ws_bytes < need) return RHQR_ENOMEM;
  RHQR_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(rhqr_info), st));
  if (o.alg == RHQR_ALG_LEFT) {
    return left_factor(s->view, W, wt, n, m, ldw, o.scaling, U, ldu, S, lds, T, R, o.want_Q ? Q : nullptr, ldq, ws,
                       ws_bytes, info, st);
  }
  if (o.alg == RHQR_ALG_BLOCK) {
    return block_factor(s->view, W, wt, n, m, ldw, o.block_size, o.scaling, U, ldu, S, lds, T, R,
                        o.want_Q ? Q : nullptr, ldq, ws, ws_bytes, info, st);
  }
  Carver c(ws, ws_bytes);
  RecBuffers b;
  RHQR_TRY(carve_rec(c, s->view, n, m, wt, o, b));
  void *Qo = o.want_Q ? Q : nullptr;
  void *Uo = o.want_U ? U : nullptr;
  if (wt == RHQR_F64)
    return rec_typed<double>(s->view, (const double *)W, wt, n, m, ldw, o, (double *)Uo, ldu, S, lds, T, R,
                             (double *)Qo, ldq, b, info, st);
  return rec_typed<float>(s->view, (const float *)W, wt, n, m, ldw, o, (float *)Uo, ldu, S, lds, T, R, (float *)Qo,
                          ldq, b, info, st);
}

rhqr_status rhqr_reconstruct(rhqr_sketch s, const double *S, int64_t lds, const double *T, const double *R,
                             const double *Z, int64_t ldz, const void *W, int32_t wt, int64_t n, int32_t m,
                             int64_t ldw, void *U, int64_t ldu, void *Q, int64_t ldq, void *ws, size_t ws_bytes,
                             rhqr_stream_t stream) {
  (void)R;
  if (s == nullptr || S == nullptr || T == nullptr || Z == nullptr || W == nullptr || U == nullptr)
    return RHQR_EINVAL;
  if (!valid_dtype_hd(wt) || m < 1) return RHQR_EINVAL;
  RHQR_TRY(check_sketch_shape(s->view, n, m));
  const int64_t p = (int64_t)s->view.k + m;
  if (lds < p || ldz < p || ldw < n || ldu < n || (Q != nullptr && ldq < n)) return RHQR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Carver c(ws, ws_bytes);
  double *StZ = c.take<double>((size_t)m * m);
  double *M = c.take<double>((size_t)m * m);
  double *Gm = c.take<double>((size_t)m * m);
  char *TriT = c.take<char>(small_padded_bytes(m));
  char *GT = c.take<char>(small_padded_bytes(m));
  if (ws == nullptr || c.overflow()) return RHQR_ENOMEM;
  RHQR_TRY(m_factor(T, S, lds, Z, ldz, p, m, StZ, M, st));
  RHQR_TRY(t_u1t(T, S, lds, m, Gm, st));
  if (wt == RHQR_F64) {
    RHQR_TRY(pad_transpose<double>(M, m, 1, (double *)TriT, st));
    RHQR_TRY(pad_transpose<double>(Gm, m, 1, (double *)GT, st));
    RHQR_TRY(rows_solve_mul<double>((const double *)W, ldw, m, n - m, m, (const double *)TriT, (const double *)GT,
                                    (double *)U, ldu, (double *)Q, ldq, st));
    RHQR_TRY(top_from_s<double>(S, lds, m, (double *)U, ldu, st));
    if (Q) RHQR_TRY(rows_form_q<double>((const double *)U, ldu, 0, m, m, (const double *)GT, (double *)Q, ldq, st));
  } else {
    RHQR_TRY(pad_transpose<float>(M, m, 1, (float *)TriT, st));
    RHQR_TRY(pad_transpose<float>(Gm, m, 1, (float *)GT, st));
    RHQR_TRY(rows_solve_mul<float>((const float *)W, ldw, m, n - m, m, (const float *)TriT, (const float *)GT,
                                   (float *)U, ldu, (float *)Q, ldq, st));
    RHQR_TRY(top_from_s<float>(S, lds, m, (float *)U, ldu, st));
    if (Q) RHQR_TRY(rows_form_q<float>((const float *)U, ldu, 0, m, m, (const float *)GT, (float *)Q, ldq, st));
  }
  return RHQR_OK;
}

// ---------------------------------------------------------------------------
// RHQR-Arnoldi
// ---------------------------------------------------------------------------

rhqr_status rhqr_arnoldi_create_batch(rhqr_sketch s, int64_t n, int32_t mmax, int32_t nrhs, int32_t basis_dtype,
                                      int32_t scaling, rhqr_arnoldi *out) {
  if (out == nullptr) return RHQR_EINVAL;
  *out = nullptr;
  if (s == nullptr || mmax < 1 || nrhs < 1 || nrhs > 65535 || !valid_dtype_hd(basis_dtype) ||
      (scaling != 0 && scaling != 1))
    return RHQR_EINVAL;
  const int32_t M = mmax + 1;
  if (M > 1024) return RHQR_ENOTSUP;
  RHQR_TRY(check_sketch_shape(s->view, n, M));
  rhqr_arnoldi a = new (std::nothrow) rhqr_arnoldi_s();
  if (a == nullptr) return RHQR_ENOMEM;
  a->st.view = s->view;
  a->st.n = n;
  a->st.M = M;
  a->st.dtype = basis_dtype;
  a->st.scaling = scaling;
  a->st.j = 0;
  a->st.nrhs = nrhs;
  size_t bytes = arnoldi_state_bytes(s->view, n, M, basis_dtype, nrhs);
  if (cudaMalloc(&a->mem, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    delete a;
    return RHQR_ENOMEM;
  }
  if (arnoldi_carve(a->st, a->mem, bytes) != RHQR_OK) {
    cudaFree(a->mem);
    delete a;
    return RHQR_ENOMEM;
  }
  if (cudaMalloc((void **)&a->lsq, sizeof(double) * arnoldi_solution_scratch_doubles(M, nrhs)) != cudaSuccess) {
    (void)cudaGetLastError();
    cudaFree(a->mem);
    delete a;
    return RHQR_ENOMEM;
  }
  *out = a;
  return RHQR_OK;
}

rhqr_status rhqr_arnoldi_create(rhqr_sketch s, int64_t n, int32_t mmax, int32_t basis_dtype, int32_t scaling,
                                rhqr_arnoldi *out) {
  return rhqr_arnoldi_create_batch(s, n, mmax, 1, basis_dtype, scaling, out);
}

rhqr_status rhqr_arnoldi_destroy(rhqr_arnoldi a) {
  if (a == nullptr) return RHQR_OK;
  cudaError_t e = cudaFree(a->mem);
  cudaError_t e2 = cudaFree(a->lsq);
  delete a;
  return (e == cudaSuccess && e2 == cudaSuccess) ? RHQR_OK : RHQR_ECUDA;
}

rhqr_status rhqr_arnoldi_begin(rhqr_arnoldi a, const void *r0, double *h0, void *q1, rhqr_info *info,
                               rhqr_stream_t stream) {
  if (a == nullptr || r0 == nullptr || h0 == nullptr || info == nullptr) return RHQR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  RHQR_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(rhqr_info) * a->st.nrhs, st));
  return arnoldi_begin(a->st, r0, h0, q1, info, st);
}

rhqr_status rhqr_arnoldi_step(rhqr_arnoldi a, const void *w, double *h, void *q_next, rhqr_info *info,
                              rhqr_stream_t stream) {
  if (a == nullptr || w == nullptr || h == nullptr || info == nullptr) return RHQR_EINVAL;
  if (a->st.j < 1 || a->st.j >= a->st.M) return RHQR_EINVAL;
  return arnoldi_step(a->st, w, h, q_next, info, (cudaStream_t)stream);
}

rhqr_status rhqr_arnoldi_solution_x(rhqr_arnoldi a, const double *H, int64_t ldh, int32_t m, const double *h0,
                                    const void *x0, void *x, int32_t xdt, double *y, double *res,
                                    rhqr_stream_t stream) {
  if (a == nullptr || H == nullptr || h0 == nullptr || y == nullptr || res == nullptr) return RHQR_EINVAL;
  if (x != nullptr && x0 == nullptr) return RHQR_EINVAL;
  return arnoldi_solution(a->st, a->lsq, H, ldh, m, h0, x0, x, xdt, y, res, (cudaStream_t)stream);
}

rhqr_status rhqr_arnoldi_solution(rhqr_arnoldi a, const double *H, int64_t ldh, int32_t m, const double *h0,
                                  const void *x0, void *x, double *y, double *res, rhqr_stream_t stream) {
  if (a == nullptr) return RHQR_EINVAL;
  return rhqr_arnoldi_solution_x(a, H, ldh, m, h0, x0, x, a->st.dtype, y, res, stream);
}

rhqr_status rhqr_arnoldi_export(rhqr_arnoldi a, void *U, int64_t ldu, double *S, int64_t lds, double *T,
                                int32_t *count, rhqr_stream_t stream) {
  if (a == nullptr) return RHQR_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const ArnoldiState &A = a->st;
  const int64_t p = (int64_t)A.view.k + A.M;
  size_t es = dtype_size(A.dtype);
  const int32_t B = A.nrhs;
  if (U != nullptr) {
    if (ldu < A.n) return RHQR_EINVAL;
    RHQR_CUDA_TRY(cudaMemcpy2DAsync(U, ldu * es, A.U, A.ldu * es, A.n * es, (size_t)A.M * B, cudaMemcpyDeviceToDevice,
                                    st));
    RHQR_TRY(arnoldi_scale_copy(A, U, ldu, st));
  }
  if (S != nullptr) {
    if (lds < p) return RHQR_EINVAL;
    RHQR_CUDA_TRY(
        cudaMemcpy2DAsync(S, lds * 8, A.S, A.lds * 8, p * 8, (size_t)A.M * B, cudaMemcpyDeviceToDevice, st));
  }
  if (T != nullptr)
    RHQR_CUDA_TRY(cudaMemcpyAsync(T, A.T, sizeof(double) * A.M * A.M * B, cudaMemcpyDeviceToDevice, st));
  if (count != nullptr) *count = A.j;
  return RHQR_OK;
}

}  // extern "C"
