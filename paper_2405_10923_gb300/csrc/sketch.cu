// RHSketch (Algorithm 1) on the GPU: Z = Psi_m X = [X_{1:m}; Omega X_{m+1:n}].
//
// SRHT (Section 2.3, Lemma "srht"): Omega_full x = sqrt(N/k) P H D x.  Here the
// signs are applied exactly, the unnormalised transform H_p is computed, the
// k sampled rows are kept and the result is scaled once by
// sqrt(N/k) / sqrt(N) = 1/sqrt(k).  The transform of length N = N1 * N2 uses the
// Kronecker structure H_N = H_{N1} (x) H_{N2} of the Sylvester order:
//   stage A: each row block of N2 entries is transformed in shared memory and
//            only the entries at the sampled in-block positions are kept;
//   stage B: each sampled row r = i1 * N2 + i2 sums its N1 stage-A values with
//            the signs (-1)^popcount(i1 & j1) (in float64, fixed order).
// Gaussian (Section 2.3): Omega = G / sqrt(k); split-K tiled product with
// float64 (or float32 within a K-chunk) accumulation and a fixed-order float64
// reduction of the chunk partials.
#include "common.cuh"
#include "fwht.cuh"
#include "sketch.cuh"

namespace rhqr {

// ---------------------------------------------------------------------------
// top block copy: Z[i, c] = X[i, c], i < m
// ---------------------------------------------------------------------------
template <class T>
__global__ void copy_top_kernel(const T *X, int64_t ldx, int32_t m, int32_t c, double *Z, int64_t ldz) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * c) return;
  int64_t col = idx / m, i = idx - col * m;
  Z[col * ldz + i] = to_f64<T>(X[col * ldx + i]);
}

// ---------------------------------------------------------------------------
// SRHT stage A: block (j1, col) transforms rows [j1*N2, (j1+1)*N2) of the
// column (rows < m and >= n read as zero, signs applied) and writes the values
// at the d2 sampled in-block positions to Y[(col * N1 + j1) * d2 + slot].
// ---------------------------------------------------------------------------
// Rows of the column held by X: global rows [first, end) at X[i - first], in
// the segments seg0, seg0 + 1, ... (the whole column: first 0, end n, seg0 0;
// a row shard of a distributed matrix: its own rows and segments).
struct RowWindow {
  int64_t first, end;
  int32_t seg0;
};

template <class T>
__global__ void srht_stage_a_kernel(const T *X, int64_t ldx, RowWindow win, int32_t m, const uint32_t *sign_bits,
                                    int32_t N2, int32_t N1, const int32_t *i2_list, int32_t d2, T *Y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *v = reinterpret_cast<T *>(smem_raw);
  const int j1 = blockIdx.x, col = blockIdx.y;
  const T *x = X + (int64_t)col * ldx;
  const int64_t row0 = (int64_t)(win.seg0 + j1) * N2;
  for (int t = threadIdx.x; t < N2; t += blockDim.x) {
    int64_t i = row0 + t;
    T val = T(0);
    if (i >= m && i >= win.first && i < win.end) {
      val = x[i - win.first];
      if ((sign_bits[i >> 5] >> (i & 31)) & 1u) val = -val;
    }
    v[t] = val;
  }
  __syncthreads();
  for (int h = 1; h < N2; h <<= 1) {
    for (int t = threadIdx.x; t < (N2 >> 1); t += blockDim.x) {
      int i = (t / h) * (2 * h) + (t % h);
      T a = v[i], b = v[i + h];
      v[i] = a + b;
      v[i + h] = a - b;
    }
    __syncthreads();
  }
  T *y = Y + ((int64_t)col * N1 + j1) * d2;
  for (int s = threadIdx.x; s < d2; s += blockDim.x) y[s] = v[i2_list[s]];
}

// SRHT stage A for segments of 512 .. 8192 entries: N2 / 16 threads, the
// column's entries loaded straight into registers (coalesced, signs and the
// zero rows applied on the way), transformed by fwht_segment, the sampled
// in-block positions written out.
template <class T, int LOGN2>
__global__ void __launch_bounds__(1 << (LOGN2 - 4)) srht_stage_a_fwht_kernel(const T *X, int64_t ldx, RowWindow win,
                                                                             int32_t m, const uint32_t *sign_bits,
                                                                             int32_t N1, const int32_t *i2_list,
                                                                             int32_t d2, T *Y) {
  constexpr int N2 = 1 << LOGN2, NT = N2 / 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *buf = reinterpret_cast<T *>(smem_raw);
  const int j1 = blockIdx.x, col = blockIdx.y, t = threadIdx.x;
  const T *x = X + (int64_t)col * ldx;
  const int64_t row0 = (int64_t)(win.seg0 + j1) * N2;
  T v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int64_t i = row0 + r * NT + t;
    T val = T(0);
    if (i >= m && i >= win.first && i < win.end) {
      val = x[i - win.first];
      if ((sign_bits[i >> 5] >> (i & 31)) & 1u) val = -val;
    }
    v[r] = val;
  }
  fwht_segment<T, LOGN2>(v, buf);
  T *y = Y + ((int64_t)col * N1 + j1) * d2;
  for (int s = t; s < d2; s += NT) y[s] = buf[i2_list[s]];
}

template <class T, int LOGN2>
static rhqr_status launch_stage_a_fwht(dim3 grid, const T *X, int64_t ldx, RowWindow win, int32_t m,
                                       const SketchView &s, T *Y, cudaStream_t st) {
  const size_t smem = sizeof(T) << LOGN2;
  if (smem > 48 * 1024)
    RHQR_CUDA_TRY(cudaFuncSetAttribute(srht_stage_a_fwht_kernel<T, LOGN2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  srht_stage_a_fwht_kernel<T, LOGN2><<<grid, 1 << (LOGN2 - 4), smem, st>>>(X, ldx, win, m, s.sign_bits, grid.x,
                                                                            s.i2_list, s.d2, Y);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

// SRHT stage B: Z[m + r, col] = (1/sqrt k) sum_{j1} (-1)^popc(i1_r & j1) Y[col, j1, slot_r],
// one warp per sampled row (lane l adds j1 = l, l + 32, ...; fixed-order tree).
template <class T>
__global__ void srht_stage_b_kernel(const T *Y, int32_t N1, int32_t d2, const int32_t *sample_i1,
                                    const int32_t *sample_slot, int32_t k, int32_t m, double scale, double *Z,
                                    int64_t ldz, int32_t seg0) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int col = blockIdx.y;
  if (r >= k) return;
  const int i1 = sample_i1[r], slot = sample_slot[r];
  const T *y = Y + (int64_t)col * N1 * d2 + slot;
  double acc = 0.0;
  for (int j1 = lane; j1 < N1; j1 += 32) {
    const double t = to_f64<T>(y[(int64_t)j1 * d2]);
    acc += (__popc(i1 & (seg0 + j1)) & 1) ? -t : t;
  }
  acc = warp_sum(acc);
  if (lane == 0) Z[(int64_t)col * ldz + m + r] = acc * scale;
}

// ---------------------------------------------------------------------------
// Gaussian split-K product: part[chunk][col][r] = sum_{kk in chunk} G[r, m+kk] X[m+kk, col]
// Tile 64 (r) x 64 (col) x 32 (kk), 256 threads, 4 x 4 outputs per thread.
// ---------------------------------------------------------------------------
constexpr int GBM = 64, GBN = 64, GBK = 32;

template <class TG, class TX, class TA>
__global__ void __launch_bounds__(256) gauss_gemm_kernel(const TG *G, int64_t ldg, const TX *X, int64_t ldx,
                                                         int64_t n, int32_t m, int32_t k, int32_t c,
                                                         int64_t chunk_len, double *part) {
  __shared__ TA Gs[GBK][GBM + 1];
  __shared__ TA Xs[GBK][GBN + 1];
  const int rt = blockIdx.x, ct = blockIdx.y, chunk = blockIdx.z;
  const int r0 = rt * GBM, c0 = ct * GBN;
  const int64_t K = n - m;
  const int64_t kb = (int64_t)chunk * chunk_len;
  const int64_t ke = min(K, kb + chunk_len);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads
  TA acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = TA(0);
  for (int64_t k0 = kb; k0 < ke; k0 += GBK) {
    // load G tile: 64 rows x 32 kk (row-major G, kk contiguous)
    for (int e = threadIdx.x; e < GBM * GBK; e += 256) {
      int rr = e / GBK, kk = e % GBK;
      int64_t gk = k0 + kk;
      TA v = TA(0);
      if (r0 + rr < k && gk < ke) v = (TA)to_f64<TG>(G[(int64_t)(r0 + rr) * ldg + m + gk]);
      Gs[kk][rr] = v;
    }
    // load X tile: 32 kk x 64 cols (column-major X, kk contiguous)
    for (int e = threadIdx.x; e < GBN * GBK; e += 256) {
      int cc = e / GBK, kk = e % GBK;
      int64_t gk = k0 + kk;
      TA v = TA(0);
      if (c0 + cc < c && gk < ke) v = (TA)to_f64<TX>(X[(int64_t)(c0 + cc) * ldx + m + gk]);
      Xs[kk][cc] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < GBK; ++kk) {
      TA g[4], x[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) g[a] = Gs[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) x[b] = Xs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += g[a] * x[b];
    }
    __syncthreads();
  }
  double *p = part + (int64_t)chunk * c * k;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int r = r0 + ty + 16 * a, cc = c0 + tx + 16 * b;
      if (r < k && cc < c) p[(int64_t)cc * k + r] = (double)acc[a][b];
    }
}

// Z[m + r, col] = scale * sum_chunk part[chunk][col][r]  (fixed order)
__global__ void reduce_chunks_kernel(const double *part, int32_t nchunk, int32_t k, int32_t c, int32_t m,
                                     double scale, double *Z, int64_t ldz) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)k * c) return;
  double acc = 0.0;
  for (int ch = 0; ch < nchunk; ++ch) acc += part[(int64_t)ch * k * c + idx];
  int64_t col = idx / k, r = idx - col * k;
  Z[col * ldz + m + r] = acc * scale;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static int gauss_chunks(int64_t K, int32_t k, int32_t c) {
  int64_t tiles = ceil_div(k, GBM) * ceil_div(c, GBN);
  int64_t want = std::max<int64_t>(1, (152 * 4) / std::max<int64_t>(1, tiles));
  int64_t maxc = std::max<int64_t>(1, ceil_div(K, 4 * GBK));
  return (int)std::min<int64_t>(want, maxc);
}

size_t sketch_apply_workspace_bytes(const SketchView &s, int32_t m, int32_t xt, int64_t n, int32_t c) {
  (void)m;
  (void)n;
  if (s.kind == RHQR_SKETCH_SRHT) {
    return align_up((size_t)c * s.N1 * s.d2 * dtype_size(xt), 256) + 256;
  }
  int nch = gauss_chunks(n - m, s.k, c);
  return align_up((size_t)nch * s.k * c * sizeof(double), 256) + 256;
}

// Stage B for many columns at once: one thread per (sampled row, column),
// the N1 segment values summed in order (enough threads without splitting a row).
template <class T>
__global__ void srht_stage_b_rows_kernel(const T *Y, int32_t N1, int32_t d2, const int32_t *sample_i1,
                                         const int32_t *sample_slot, int32_t k, int32_t m, double scale, double *Z,
                                         int64_t ldz, int32_t seg0) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int col = blockIdx.y;
  if (r >= k) return;
  const int i1 = sample_i1[r], slot = sample_slot[r];
  const T *y = Y + (int64_t)col * N1 * d2 + slot;
  double acc = 0.0;
  for (int j1 = 0; j1 < N1; ++j1) {
    const double t = to_f64<T>(y[(int64_t)j1 * d2]);
    acc += (__popc(i1 & (seg0 + j1)) & 1) ? -t : t;
  }
  Z[(int64_t)col * ldz + m + r] = acc * scale;
}

// Stage A over the segments seg0 .. seg0 + nseg - 1 of the window's rows,
// stage B summing them with the global segment signs: Z[m + r, col] for the
// rows in the window (the whole column, or a shard's share of the sum).
template <class TX>
static rhqr_status srht_apply(const SketchView &s, int32_t m, const TX *X, int64_t ldx, RowWindow win, int32_t nseg,
                              int32_t c, double *Z, int64_t ldz, void *ws, size_t ws_bytes, cudaStream_t st) {
  TX *Y = (TX *)ws;
  size_t need = (size_t)c * nseg * s.d2 * sizeof(TX);
  if (ws_bytes < need) return RHQR_ENOMEM;
  dim3 ga((unsigned)nseg, c);
  switch (s.N2) {
    case 8192: RHQR_TRY((launch_stage_a_fwht<TX, 13>(ga, X, ldx, win, m, s, Y, st))); break;
    case 4096: RHQR_TRY((launch_stage_a_fwht<TX, 12>(ga, X, ldx, win, m, s, Y, st))); break;
    case 2048: RHQR_TRY((launch_stage_a_fwht<TX, 11>(ga, X, ldx, win, m, s, Y, st))); break;
    case 1024: RHQR_TRY((launch_stage_a_fwht<TX, 10>(ga, X, ldx, win, m, s, Y, st))); break;
    case 512: RHQR_TRY((launch_stage_a_fwht<TX, 9>(ga, X, ldx, win, m, s, Y, st))); break;
    default: {  // short transforms: one butterfly level per step in shared memory
      size_t smem = (size_t)s.N2 * sizeof(TX);
      srht_stage_a_kernel<TX><<<ga, 512, smem, st>>>(X, ldx, win, m, s.sign_bits, s.N2, nseg, s.i2_list, s.d2, Y);
      RHQR_LAUNCH_CHECK();
    }
  }
  if (c >= 16) {  // enough (row, column) pairs to fill the GPU with one thread each
    dim3 gb((unsigned)ceil_div(s.k, 128), c);
    srht_stage_b_rows_kernel<TX><<<gb, 128, 0, st>>>(Y, nseg, s.d2, s.sample_i1, s.sample_slot, s.k, m,
                                                      1.0 / sqrt((double)s.k), Z, ldz, win.seg0);
  } else {  // few columns: a warp per sampled row
    dim3 gb((unsigned)ceil_div(s.k, 8), c);
    srht_stage_b_kernel<TX><<<gb, 256, 0, st>>>(Y, nseg, s.d2, s.sample_i1, s.sample_slot, s.k, m,
                                                 1.0 / sqrt((double)s.k), Z, ldz, win.seg0);
  }
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

template <class TX>
static rhqr_status apply_typed(const SketchView &s, int32_t m, const TX *X, int64_t n, int32_t c, int64_t ldx,
                               double *Z, int64_t ldz, void *ws, size_t ws_bytes, cudaStream_t st) {
  if (m > 0) {
    int64_t tot = (int64_t)m * c;
    copy_top_kernel<TX><<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(X, ldx, m, c, Z, ldz);
    RHQR_LAUNCH_CHECK();
  }
  if (s.kind == RHQR_SKETCH_SRHT) return srht_apply<TX>(s, m, X, ldx, RowWindow{0, n, 0}, s.N1, c, Z, ldz, ws, ws_bytes, st);
  // Gaussian
  int64_t K = n - m;
  int nch = gauss_chunks(K, s.k, c);
  size_t need = (size_t)nch * s.k * c * sizeof(double);
  if (ws_bytes < need) return RHQR_ENOMEM;
  double *part = (double *)ws;
  int64_t chunk_len = ceil_div(ceil_div(K, nch), GBK) * GBK;
  nch = (int)ceil_div(K, chunk_len);
  dim3 grid((unsigned)ceil_div(s.k, GBM), (unsigned)ceil_div(c, GBN), (unsigned)nch);
  const bool wide = sizeof(TX) == 8;
  switch (s.omega_dtype) {
    case RHQR_F64:
      if (wide)
        gauss_gemm_kernel<double, TX, double><<<grid, 256, 0, st>>>((const double *)s.G, s.ldg, X, ldx, n, m, s.k, c,
                                                                   chunk_len, part);
      else
        gauss_gemm_kernel<double, TX, float><<<grid, 256, 0, st>>>((const double *)s.G, s.ldg, X, ldx, n, m, s.k, c,
                                                                  chunk_len, part);
      break;
    case RHQR_F32:
      if (wide)
        gauss_gemm_kernel<float, TX, double><<<grid, 256, 0, st>>>((const float *)s.G, s.ldg, X, ldx, n, m, s.k, c,
                                                                  chunk_len, part);
      else
        gauss_gemm_kernel<float, TX, float><<<grid, 256, 0, st>>>((const float *)s.G, s.ldg, X, ldx, n, m, s.k, c,
                                                                 chunk_len, part);
      break;
    case RHQR_BF16:
      if (wide)
        gauss_gemm_kernel<__nv_bfloat16, TX, double><<<grid, 256, 0, st>>>((const __nv_bfloat16 *)s.G, s.ldg, X, ldx,
                                                                          n, m, s.k, c, chunk_len, part);
      else
        gauss_gemm_kernel<__nv_bfloat16, TX, float><<<grid, 256, 0, st>>>((const __nv_bfloat16 *)s.G, s.ldg, X, ldx,
                                                                         n, m, s.k, c, chunk_len, part);
      break;
    case RHQR_F16:
      if (wide)
        gauss_gemm_kernel<__half, TX, double><<<grid, 256, 0, st>>>((const __half *)s.G, s.ldg, X, ldx, n, m, s.k, c,
                                                                   chunk_len, part);
      else
        gauss_gemm_kernel<__half, TX, float><<<grid, 256, 0, st>>>((const __half *)s.G, s.ldg, X, ldx, n, m, s.k, c,
                                                                  chunk_len, part);
      break;
    default:
      return RHQR_EINVAL;
  }
  RHQR_LAUNCH_CHECK();
  int64_t tot = (int64_t)s.k * c;
  reduce_chunks_kernel<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(part, nch, s.k, c, m, 1.0 / sqrt((double)s.k),
                                                                     Z, ldz);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

// Top block of a shard's Z: Z[i, col] = X[i - row0, col] for the rows i < m
// in [row0, row0 + rows), else 0.
template <class TX>
__global__ void shard_top_kernel(const TX *X, int64_t ldx, int64_t row0, int64_t rows, int32_t m, int32_t c,
                                 double *Z, int64_t ldz) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * c) return;
  const int64_t col = idx / m, i = idx - col * m;
  Z[col * ldz + i] = (i >= row0 && i < row0 + rows) ? to_f64<TX>(X[col * ldx + (i - row0)]) : 0.0;
}

size_t sketch_rows_workspace_bytes(const SketchView &s, int32_t m, int32_t xt, int64_t row0, int64_t rows,
                                   int32_t c) {
  if (s.kind == RHQR_SKETCH_SRHT) {
    const int64_t nseg = ceil_div(rows, s.N2);
    return align_up((size_t)c * nseg * s.d2 * dtype_size(xt), 256) + 256;
  }
  const int32_t ml = (int32_t)std::min<int64_t>(std::max<int64_t>(m - row0, 0), rows);
  return sketch_apply_workspace_bytes(s, ml, xt, rows, c);
}

template <class TX>
static rhqr_status rows_typed(const SketchView &s, int32_t m, const TX *X, int64_t row0, int64_t rows, int32_t c,
                              int64_t ldx, double *Z, int64_t ldz, void *ws, size_t ws_bytes, cudaStream_t st) {
  if (s.kind == RHQR_SKETCH_SRHT) {
    const int32_t nseg = (int32_t)ceil_div(rows, s.N2);
    RHQR_TRY(srht_apply<TX>(s, m, X, ldx, RowWindow{row0, row0 + rows, (int32_t)(row0 / s.N2)}, nseg, c, Z, ldz, ws,
                            ws_bytes, st));
  } else {
    // the shard's columns of Omega_full: the operator seen from column row0
    SketchView v = s;
    v.G = (const char *)s.G + (size_t)row0 * dtype_size(s.omega_dtype);
    v.Gt = nullptr;
    const int32_t ml = (int32_t)std::min<int64_t>(std::max<int64_t>(m - row0, 0), rows);
    if (ml < rows) {
      // Z rows m .. m + k - 1 from the shard's rows ml .. rows - 1 (global row0 + ml ..)
      RHQR_TRY(apply_typed<TX>(v, ml, X, rows, c, ldx, Z + (m - ml), ldz, ws, ws_bytes, st));
    } else {
      RHQR_CUDA_TRY(cudaMemset2DAsync(Z + m, ldz * sizeof(double), 0, (size_t)s.k * sizeof(double), c, st));
    }
  }
  if (m > 0) {
    shard_top_kernel<TX><<<(unsigned)ceil_div((int64_t)m * c, 256), 256, 0, st>>>(X, ldx, row0, rows, m, c, Z, ldz);
    RHQR_LAUNCH_CHECK();
  }
  return RHQR_OK;
}

rhqr_status sketch_apply_rows_simt(const SketchView &s, int32_t m, const void *X, int32_t xt, int64_t row0,
                                   int64_t rows, int32_t c, int64_t ldx, double *Z, int64_t ldz, void *ws,
                                   size_t ws_bytes, cudaStream_t st) {
  if (xt == RHQR_F64)
    return rows_typed<double>(s, m, (const double *)X, row0, rows, c, ldx, Z, ldz, ws, ws_bytes, st);
  if (xt == RHQR_F32)
    return rows_typed<float>(s, m, (const float *)X, row0, rows, c, ldx, Z, ldz, ws, ws_bytes, st);
  return RHQR_ENOTSUP;
}

rhqr_status sketch_apply_simt(const SketchView &s, int32_t m, const void *X, int32_t xt, int64_t n, int32_t c,
                              int64_t ldx, double *Z, int64_t ldz, void *ws, size_t ws_bytes, cudaStream_t st) {
  if (xt == RHQR_F64)
    return apply_typed<double>(s, m, (const double *)X, n, c, ldx, Z, ldz, ws, ws_bytes, st);
  if (xt == RHQR_F32) return apply_typed<float>(s, m, (const float *)X, n, c, ldx, Z, ldz, ws, ws_bytes, st);
  return RHQR_ENOTSUP;
}

}  // namespace rhqr
