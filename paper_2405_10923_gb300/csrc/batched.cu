// Batched recRHQR (Algorithm 6 with refinement passes) for many independent,
// ragged tall-skinny problems with SRHT sketches.
//
// A batch plan (rhqr_batch_create) binds, once, the problems' sketches, shapes
// and data pointers, and uploads a per-problem table with the work-prefix
// offsets and workspace offsets.  rhqr_factor_batched then only enqueues
// kernels -- no host synchronisation or allocation -- so a caller can capture
// it in a CUDA graph and replay the whole batch as one graph launch.  Every
// phase is one launch covering all problems:
//   1. SRHT stage A: work item (problem, column, row block of N2 rows)
//   2. SRHT stage B and the exact top block: item (problem, column, row)
//   3. Householder QR of each problem's sketch, one CTA per problem, float64
//   4. R accumulation over passes, padded float transposes of R
//   5. row solves Q = X R^{-1}: item (problem, block of rows)
//   6. last pass: T from the Woodbury identity, S and R outputs, info
// Items are mapped to problems by a binary search over the prefix offsets.
#include <algorithm>
#include <new>
#include <vector>

#include "common.cuh"
#include "fwht.cuh"
#include "sketch.cuh"

namespace rhqr {

const SketchView *sketch_view_of(rhqr_sketch s);

struct BatchProb {
  int64_t n, ldx, ldq, lds;
  int32_t m, k, N1, N2, d2, mp;
  const void *W;
  void *Q;
  double *S, *T, *R;
  const uint32_t *signs;
  const int32_t *i2, *si1, *sslot;
  int64_t off_Z, off_Y, off_beta, off_Rp, off_Racc, off_Rtmp, off_SS, off_TriT;
  int64_t a_begin, b_begin;
  int64_t s_begin[3];  // first row-block item of the solve, for 32 / 64 / 128 rows per block
};

// Row-block sizes of the batched solve among which the tuner chooses.
#define RB_INDEX(rb) ((rb) == 32 ? 0 : (rb) == 64 ? 1 : 2)

// Problem owning work item `item` of a phase: the last problem whose first item
// of that phase is <= item (binary search over the prefix offsets).
template <class F>
__device__ __forceinline__ int find_prob_by(const BatchProb *P, int count, int64_t item, F first) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (first(P[mid]) <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int find_prob_a(const BatchProb *P, int count, int64_t item) {
  return find_prob_by(P, count, item, [](const BatchProb &b) { return b.a_begin; });
}
__device__ __forceinline__ int find_prob_b(const BatchProb *P, int count, int64_t item) {
  return find_prob_by(P, count, item, [](const BatchProb &b) { return b.b_begin; });
}
__device__ __forceinline__ int find_prob_rows(const BatchProb *P, int count, int64_t item, int rb) {
  const int ix = RB_INDEX(rb);
  return find_prob_by(P, count, item, [ix](const BatchProb &b) { return b.s_begin[ix]; });
}

// ---- 1. SRHT stage A (per (problem, column, block)) -------------------------
template <class T>
__global__ void __launch_bounds__(1024) b_srht_a_kernel(const BatchProb *P, int count, int pass, char *ws, int64_t items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *v = reinterpret_cast<T *>(smem_raw);
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int pi = find_prob_a(P, count, item);
    const BatchProb &B = P[pi];
    const int64_t local = item - B.a_begin;
    const int col = (int)(local / B.N1), j1 = (int)(local % B.N1);
    const T *X = pass == 0 ? (const T *)B.W : (const T *)B.Q;
    const int64_t ldx = pass == 0 ? B.ldx : B.ldq;
    const T *x = X + (int64_t)col * ldx;
    const int64_t row0 = (int64_t)j1 * B.N2;
    __syncthreads();
    for (int t = threadIdx.x; t < B.N2; t += blockDim.x) {
      int64_t i = row0 + t;
      T val = T(0);
      if (i >= B.m && i < B.n) {
        val = x[i];
        if ((B.signs[i >> 5] >> (i & 31)) & 1u) val = -val;
      }
      v[t] = val;
    }
    __syncthreads();
    for (int h = 1; h < B.N2; h <<= 1) {
      for (int t = threadIdx.x; t < (B.N2 >> 1); t += blockDim.x) {
        int i = (t / h) * (2 * h) + (t % h);
        T a = v[i], b = v[i + h];
        v[i] = a + b;
        v[i + h] = a - b;
      }
      __syncthreads();
    }
    T *Y = reinterpret_cast<T *>(ws + B.off_Y) + ((int64_t)col * B.N1 + j1) * B.d2;
    for (int s = threadIdx.x; s < B.d2; s += blockDim.x) Y[s] = v[B.i2[s]];
  }
}

// The same for batches whose problems all have 8192-entry segments (every
// N >= 8192): 512 threads, the register / shuffle transform of fwht.cuh.
template <class T>
__global__ void __launch_bounds__(512) b_srht_a_fwht_kernel(const BatchProb *P, int count, int pass, char *ws,
                                                            int64_t items) {
  constexpr int NT = 512;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *buf = reinterpret_cast<T *>(smem_raw);
  const int t = threadIdx.x;
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int pi = find_prob_a(P, count, item);
    const BatchProb &B = P[pi];
    const int64_t local = item - B.a_begin;
    const int col = (int)(local / B.N1), j1 = (int)(local % B.N1);
    const T *X = pass == 0 ? (const T *)B.W : (const T *)B.Q;
    const int64_t ldx = pass == 0 ? B.ldx : B.ldq;
    const T *x = X + (int64_t)col * ldx;
    const int64_t row0 = (int64_t)j1 * 8192;
    T v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int64_t i = row0 + r * NT + t;
      T val = T(0);
      if (i >= B.m && i < B.n) {
        val = x[i];
        if ((B.signs[i >> 5] >> (i & 31)) & 1u) val = -val;
      }
      v[r] = val;
    }
    __syncthreads();  // the previous item's samples are read before buf is rewritten
    fwht_segment<T, 13>(v, buf);
    T *Y = reinterpret_cast<T *>(ws + B.off_Y) + ((int64_t)col * B.N1 + j1) * B.d2;
    for (int s2 = t; s2 < B.d2; s2 += NT) Y[s2] = buf[B.i2[s2]];
  }
}

// ---- 2. SRHT stage B + exact top block (per (problem, column, sketch row)) --
template <class T>
__global__ void b_srht_b_kernel(const BatchProb *P, int count, int pass, char *ws, int64_t items) {
  for (int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; item < items;
       item += (int64_t)gridDim.x * blockDim.x) {
    const int pi = find_prob_b(P, count, item);
    const BatchProb &B = P[pi];
    const int64_t local = item - B.b_begin;
    const int p = B.k + B.m;
    const int col = (int)(local / p), r = (int)(local % p);
    double *Z = reinterpret_cast<double *>(ws + B.off_Z);
    if (r < B.m) {  // exact top block
      const T *X = pass == 0 ? (const T *)B.W : (const T *)B.Q;
      const int64_t ldx = pass == 0 ? B.ldx : B.ldq;
      Z[(int64_t)col * p + r] = (double)X[(int64_t)col * ldx + r];
    } else {
      const int rr = r - B.m;
      const int i1 = B.si1[rr], slot = B.sslot[rr];
      const T *y = reinterpret_cast<const T *>(ws + B.off_Y) + (int64_t)col * B.N1 * B.d2 + slot;
      double acc = 0.0;
      for (int j1 = 0; j1 < B.N1; ++j1) {
        double t = (double)y[(int64_t)j1 * B.d2];
        acc += (__popc(i1 & j1) & 1) ? -t : t;
      }
      Z[(int64_t)col * p + r] = acc * rsqrt((double)B.k);
    }
  }
}

// ---- 3. Householder QR of Z (one CTA per problem, in place) ----------------
__global__ void __launch_bounds__(512) b_hqr_kernel(const BatchProb *P, int count, char *ws, int scaling,
                                                    rhqr_info *info) {
  __shared__ double red[32];
  __shared__ double sh[4];
  const int pi = blockIdx.x;
  if (pi >= count) return;
  const BatchProb &B = P[pi];
  const int p = B.k + B.m, m = B.m;
  double *Z = reinterpret_cast<double *>(ws + B.off_Z);
  double *beta = reinterpret_cast<double *>(ws + B.off_beta);
  double *Rp = reinterpret_cast<double *>(ws + B.off_Rp);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < m; ++j) {
    double s = 0.0;
    for (int i = j + threadIdx.x; i < p; i += blockDim.x) s += Z[(int64_t)j * p + i] * Z[(int64_t)j * p + i];
    s = block_sum(s, red);
    const double rho = sqrt(s), a = Z[(int64_t)j * p + j];
    if (!isfinite(rho) || !isfinite(a) || rho == 0.0) {
      if (threadIdx.x == 0) set_status(info + pi, rho == 0.0 ? RHQR_EBREAKDOWN : RHQR_ENONFINITE, j);
      return;
    }
    const double sigma = a < 0.0 ? -1.0 : 1.0, g = a + sigma * rho;
    const double div = scaling == 0 ? g : sqrt(rho * (rho + fabs(a)));
    if (threadIdx.x == 0) {
      beta[j] = scaling == 0 ? 1.0 + fabs(a) / rho : 1.0;
      sh[0] = beta[j];
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      Rp[(int64_t)j * m + i] = i < j ? Z[(int64_t)j * p + i] : (i == j ? -sigma * rho : 0.0);
    __syncthreads();
    for (int i = j + threadIdx.x; i < p; i += blockDim.x)
      Z[(int64_t)j * p + i] = (i == j) ? g / div : Z[(int64_t)j * p + i] / div;
    __syncthreads();
    const double bj = sh[0];
    for (int c = j + 1 + wid; c < m; c += nw) {
      double d = 0.0;
      for (int i = j + lane; i < p; i += 32) d += Z[(int64_t)j * p + i] * Z[(int64_t)c * p + i];
      d = warp_sum(d) * bj;
      for (int i = j + lane; i < p; i += 32) Z[(int64_t)c * p + i] -= Z[(int64_t)j * p + i] * d;
    }
    __syncthreads();
  }
}

// ---- 4. R accumulation and padded transposes -------------------------------
// pass 0: Racc = Rp; else Racc = Rp Racc.  TriT (mp x mp in W's dtype, row l
// contiguous, identity on the padding) = Rp.
template <class T>
__global__ void b_racc_kernel(const BatchProb *P, int count, char *ws, int pass) {
  const int pi = blockIdx.x;
  if (pi >= count) return;
  const BatchProb &B = P[pi];
  const int m = B.m, mp = B.mp;
  const double *Rp = reinterpret_cast<const double *>(ws + B.off_Rp);
  double *Racc = reinterpret_cast<double *>(ws + B.off_Racc);
  double *Rt = reinterpret_cast<double *>(ws + B.off_Rtmp);
  T *TriT = reinterpret_cast<T *>(ws + B.off_TriT);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int j = e / m, i = e % m;
    double acc = 0.0;
    if (pass == 0) acc = Rp[e];
    else if (i <= j)
      for (int l = i; l <= j; ++l) acc += Rp[(int64_t)l * m + i] * Racc[(int64_t)j * m + l];
    Rt[e] = acc;
  }
  for (int e = threadIdx.x; e < mp * mp; e += blockDim.x) {
    int l = e / mp, j = e % mp;
    double v = (l < m && j < m) ? (l <= j ? Rp[(int64_t)j * m + l] : 0.0) : (l == j ? 1.0 : 0.0);
    TriT[e] = (T)v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) Racc[e] = Rt[e];
}

// ---- 5. row solves Q = X Tri^{-1} (block of RB rows of one problem) --------
// One thread owns one row (an independent forward substitution); the row sits
// in shared memory column-major in the block and is solved in panels of 32.
template <class T>
__device__ __forceinline__ void b_load_panel(const T *p, T (&r)[32]);
template <>
__device__ __forceinline__ void b_load_panel<float>(const float *p, float (&r)[32]) {
  const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float4 v = __ldg(q + i);
    r[4 * i] = v.x;
    r[4 * i + 1] = v.y;
    r[4 * i + 2] = v.z;
    r[4 * i + 3] = v.w;
  }
}
template <>
__device__ __forceinline__ void b_load_panel<double>(const double *p, double (&r)[32]) {
  const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    double2 v = __ldg(q + i);
    r[2 * i] = v.x;
    r[2 * i + 1] = v.y;
  }
}

template <class T, int RB>
__global__ void __launch_bounds__(RB) b_solve_kernel(const BatchProb *P, int count, char *ws, int pass,
                                                     int64_t items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *xs = reinterpret_cast<T *>(smem_raw);
  const int t = threadIdx.x;
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int pi = find_prob_rows(P, count, item, RB);
    const BatchProb &B = P[pi];
    const int64_t blk = item - B.s_begin[RB_INDEX(RB)];
    const int m = B.m, mp = B.mp;
    const int64_t i = blk * RB + t;
    const bool live = i < B.n;
    const T *X = pass == 0 ? (const T *)B.W : (const T *)B.Q;
    const int64_t ldx = pass == 0 ? B.ldx : B.ldq;
    const T *TriT = reinterpret_cast<const T *>(ws + B.off_TriT);
    for (int j = 0; j < mp; ++j) xs[j * RB + t] = (live && j < m) ? X[(int64_t)j * ldx + i] : T(0);
    for (int J0 = 0; J0 < mp; J0 += 32) {
      T acc[32];
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) acc[jj] = xs[(J0 + jj) * RB + t];
      for (int l = 0; l < J0; ++l) {
        T r[32];
        b_load_panel<T>(TriT + (int64_t)l * mp + J0, r);
        const T yl = xs[l * RB + t];
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) acc[jj] -= yl * r[jj];
      }
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        T r[32];
        b_load_panel<T>(TriT + (int64_t)(J0 + jj) * mp + J0, r);
        acc[jj] = acc[jj] / r[jj];
#pragma unroll
        for (int q = jj + 1; q < 32; ++q) acc[q] -= acc[jj] * r[q];
      }
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) xs[(J0 + jj) * RB + t] = acc[jj];
    }
    if (live) {
      T *Q = (T *)B.Q;
      for (int j = 0; j < m; ++j) Q[(int64_t)j * B.ldq + i] = xs[j * RB + t];
    }
  }
}

// ---- 6. outputs of the last pass: S, R, T (Woodbury), info -----------------
__global__ void b_finish_kernel(const BatchProb *P, int count, char *ws, int passes, rhqr_info *info) {
  const int pi = blockIdx.x;
  if (pi >= count) return;
  const BatchProb &B = P[pi];
  const int p = B.k + B.m, m = B.m;
  const double *Z = reinterpret_cast<const double *>(ws + B.off_Z);  // Householder vectors (in place)
  const double *beta = reinterpret_cast<const double *>(ws + B.off_beta);
  const double *Racc = reinterpret_cast<const double *>(ws + B.off_Racc);
  double *SS = reinterpret_cast<double *>(ws + B.off_SS);
  // S: the Householder vectors (zero above the diagonal)
  for (int64_t e = threadIdx.x; e < (int64_t)p * m; e += blockDim.x) {
    int j = (int)(e / p), i = (int)(e % p);
    B.S[(int64_t)j * B.lds + i] = i < j ? 0.0 : Z[e];
  }
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) B.R[e] = Racc[e];
  // SS[i, j] = s_i . s_j (i < j), then T column by column (one warp per column)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int pr = wid; pr < m * m; pr += nw) {
    int j = pr / m, i = pr % m;
    if (i >= j) continue;
    double d = 0.0;
    for (int r = j + lane; r < p; r += 32) d += Z[(int64_t)i * p + r] * Z[(int64_t)j * p + r];
    d = warp_sum(d);
    if (lane == 0) SS[(int64_t)j * m + i] = d;
  }
  __syncthreads();
  for (int j = wid; j < m; j += nw) {
    double *t = B.T + (int64_t)j * m;
    for (int i = j + 1 + lane; i < m; i += 32) t[i] = 0.0;
    if (lane == 0) t[j] = beta[j];
    __syncwarp();
    for (int i = j - 1; i >= 0; --i) {
      double d = 0.0;
      for (int l = i + 1 + lane; l <= j; l += 32) d += SS[(int64_t)l * m + i] * t[l];
      d = warp_sum(d);
      if (lane == 0) t[i] = -beta[i] * d;
      __syncwarp();
    }
  }
  if (threadIdx.x == 0 && info[pi].status == RHQR_OK) info[pi].passes_done = passes;
}

}  // namespace rhqr

using namespace rhqr;

struct rhqr_batch_s {
  int32_t count, wt, passes, scaling;
  std::vector<BatchProb> host;
  BatchProb *dev;
  size_t ws_bytes;
  int64_t itemsA, itemsB, itemsS[3];
  int32_t maxN2, minN2, maxmp;
  // launch shapes (set by the tuner): stage-A threads, solve rows per block,
  // solve grid cap (0 = one block per row block)
  int32_t a_threads, solve_rb, solve_cap;
};

namespace rhqr {

static const int32_t kAThreads[] = {128, 256, 512, 1024};
static const int32_t kSolveRB[] = {32, 64, 128};
static const int32_t kSolveCap[] = {0, 152 * 16, 152 * 4};

template <class T>
static rhqr_status batch_set_smem(size_t smemA, size_t smemS32) {
  RHQR_CUDA_TRY(cudaFuncSetAttribute(b_srht_a_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemA));
  RHQR_CUDA_TRY(cudaFuncSetAttribute(b_solve_kernel<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smemS32));
  RHQR_CUDA_TRY(cudaFuncSetAttribute(b_solve_kernel<T, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(2 * smemS32)));
  RHQR_CUDA_TRY(cudaFuncSetAttribute(b_solve_kernel<T, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(4 * smemS32)));
  return RHQR_OK;
}

template <class T>
static rhqr_status batch_stage_a(const rhqr_batch_s *b, char *w, int pass, int threads, cudaStream_t st) {
  if (b->minN2 == 8192 && b->maxN2 == 8192) {
    const size_t smem = 8192 * sizeof(T);
    RHQR_CUDA_TRY(cudaFuncSetAttribute(b_srht_a_fwht_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    const unsigned g = (unsigned)std::min<int64_t>(b->itemsA, 152 * 4);
    b_srht_a_fwht_kernel<T><<<g, 512, smem, st>>>(b->dev, b->count, pass, w, b->itemsA);
    RHQR_LAUNCH_CHECK();
    return RHQR_OK;
  }
  const unsigned g = (unsigned)std::min<int64_t>(b->itemsA, 152 * 2048 / threads * 2);
  b_srht_a_kernel<T><<<g, threads, (size_t)b->maxN2 * sizeof(T), st>>>(b->dev, b->count, pass, w, b->itemsA);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

template <class T>
static rhqr_status batch_solve(const rhqr_batch_s *b, char *w, int pass, int rb, int cap, cudaStream_t st) {
  const int ix = RB_INDEX(rb);
  const int64_t items = b->itemsS[ix];
  const unsigned g = (unsigned)(cap > 0 ? std::min<int64_t>(items, cap) : std::min<int64_t>(items, INT32_MAX));
  const size_t smem = (size_t)b->maxmp * rb * sizeof(T);
  if (rb == 32) b_solve_kernel<T, 32><<<g, 32, smem, st>>>(b->dev, b->count, w, pass, items);
  else if (rb == 64) b_solve_kernel<T, 64><<<g, 64, smem, st>>>(b->dev, b->count, w, pass, items);
  else b_solve_kernel<T, 128><<<g, 128, smem, st>>>(b->dev, b->count, w, pass, items);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

template <class T>
static rhqr_status batch_run(const rhqr_batch_s *b, char *w, rhqr_info *info, cudaStream_t st) {
  const int cnt = b->count;
  RHQR_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(rhqr_info) * cnt, st));
  const unsigned gB = (unsigned)std::min<int64_t>(ceil_div(b->itemsB, 256), 152 * 32);
  for (int pass = 0; pass < b->passes; ++pass) {
    {
      PhaseScope ps(PH_SKETCH, st);
      RHQR_TRY(batch_stage_a<T>(b, w, pass, b->a_threads, st));
      b_srht_b_kernel<T><<<gB, 256, 0, st>>>(b->dev, cnt, pass, w, b->itemsB);
      RHQR_LAUNCH_CHECK();
    }
    {
      PhaseScope ps(PH_HQR, st);
      b_hqr_kernel<<<cnt, 512, 0, st>>>(b->dev, cnt, w, b->scaling, info);
      RHQR_LAUNCH_CHECK();
      b_racc_kernel<T><<<cnt, 256, 0, st>>>(b->dev, cnt, w, pass);
      RHQR_LAUNCH_CHECK();
    }
    {
      PhaseScope ps(PH_SOLVE, st);
      RHQR_TRY(batch_solve<T>(b, w, pass, b->solve_rb, b->solve_cap, st));
    }
  }
  PhaseScope ps(PH_TFACTOR, st);
  b_finish_kernel<<<cnt, 256, 0, st>>>(b->dev, cnt, w, b->passes, info);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

// Mean time (ms) of `reps` launches of fn on st, after one untimed launch.
template <class F>
static rhqr_status time_launches(F fn, int reps, cudaStream_t st, float *ms) {
  cudaEvent_t e0, e1;
  RHQR_CUDA_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return RHQR_ECUDA;
  }
  rhqr_status r = fn();
  if (r == RHQR_OK && cudaEventRecord(e0, st) != cudaSuccess) r = RHQR_ECUDA;
  for (int i = 0; i < reps && r == RHQR_OK; ++i) r = fn();
  if (r == RHQR_OK && cudaEventRecord(e1, st) != cudaSuccess) r = RHQR_ECUDA;
  if (r == RHQR_OK && cudaEventSynchronize(e1) != cudaSuccess) r = RHQR_ECUDA;
  if (r == RHQR_OK && cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) r = RHQR_ECUDA;
  if (r == RHQR_OK) *ms /= (float)reps;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return r;
}

template <class T>
static rhqr_status batch_tune(rhqr_batch_s *b, char *w, rhqr_info *info, int reps, cudaStream_t st) {
  RHQR_TRY(batch_run<T>(b, w, info, st));  // fills the workspace with a valid pass
  float best = 1e30f;
  for (int32_t th : kAThreads) {
    float ms = 0.f;
    RHQR_TRY(time_launches([&] { return batch_stage_a<T>(b, w, 0, th, st); }, reps, st, &ms));
    if (ms < best) {
      best = ms;
      b->a_threads = th;
    }
  }
  best = 1e30f;
  for (int32_t rb : kSolveRB)
    for (int32_t cap : kSolveCap) {
      float ms = 0.f;
      RHQR_TRY(time_launches([&] { return batch_solve<T>(b, w, 0, rb, cap, st); }, reps, st, &ms));
      if (ms < best) {
        best = ms;
        b->solve_rb = rb;
        b->solve_cap = cap;
      }
    }
  return RHQR_OK;
}

}  // namespace rhqr

extern "C" {

rhqr_status rhqr_batch_create(int32_t count, const rhqr_sketch *s, const void *const *W, int32_t wt,
                              const int64_t *n, const int32_t *m, const int64_t *ldw, const rhqr_opts *opts,
                              void *const *Q, const int64_t *ldq, double *const *S, const int64_t *lds,
                              double *const *T, double *const *R, rhqr_batch *out) {
  if (out == nullptr) return RHQR_EINVAL;
  *out = nullptr;
  if (count < 1 || s == nullptr || W == nullptr || n == nullptr || m == nullptr || ldw == nullptr || Q == nullptr ||
      ldq == nullptr || S == nullptr || lds == nullptr || T == nullptr || R == nullptr)
    return RHQR_EINVAL;
  if (wt != RHQR_F64 && wt != RHQR_F32) return RHQR_EINVAL;
  rhqr_opts o;
  if (opts) o = *opts;
  else rhqr_default_opts(&o);
  if (o.passes < 1 || o.passes > 16 || (o.scaling != 0 && o.scaling != 1)) return RHQR_EINVAL;
  rhqr_batch b = new (std::nothrow) rhqr_batch_s();
  if (b == nullptr) return RHQR_ENOMEM;
  b->count = count;
  b->wt = wt;
  b->passes = o.passes;
  b->scaling = o.scaling;
  b->a_threads = 512;
  b->solve_rb = 64;
  b->solve_cap = 0;
  b->dev = nullptr;
  b->host.resize(count);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = align_up(off, 256);
    size_t r = off;
    off += bytes;
    return (int64_t)r;
  };
  int64_t a = 0, bb = 0, sblk[3] = {0, 0, 0};
  b->maxN2 = 1;
  b->minN2 = 1 << 30;
  b->maxmp = 32;
  const size_t es = dtype_size(wt);
  for (int i = 0; i < count; ++i) {
    if (s[i] == nullptr || W[i] == nullptr || Q[i] == nullptr || S[i] == nullptr || T[i] == nullptr ||
        R[i] == nullptr) {
      delete b;
      return RHQR_EINVAL;
    }
    const SketchView &v = *sketch_view_of(s[i]);
    if (v.kind != RHQR_SKETCH_SRHT || m[i] < 1 || m[i] > 128 || n[i] <= m[i] || n[i] > v.N || m[i] > v.k ||
        ldw[i] < n[i] || ldq[i] < n[i] || lds[i] < (int64_t)v.k + m[i]) {
      delete b;
      return RHQR_EINVAL;
    }
    BatchProb &P = b->host[i];
    P.n = n[i];
    P.m = m[i];
    P.k = v.k;
    P.N1 = v.N1;
    P.N2 = v.N2;
    P.d2 = v.d2;
    P.mp = (int32_t)ceil_div(m[i], 32) * 32;
    P.ldx = ldw[i];
    P.ldq = ldq[i];
    P.lds = lds[i];
    P.W = W[i];
    P.Q = Q[i];
    P.S = S[i];
    P.T = T[i];
    P.R = R[i];
    P.signs = v.sign_bits;
    P.i2 = v.i2_list;
    P.si1 = v.sample_i1;
    P.sslot = v.sample_slot;
    const int64_t p = (int64_t)v.k + m[i];
    P.off_Z = take((size_t)p * m[i] * 8);
    P.off_Y = take((size_t)m[i] * v.N1 * v.d2 * es);
    P.off_beta = take((size_t)m[i] * 8);
    P.off_Rp = take((size_t)m[i] * m[i] * 8);
    P.off_Racc = take((size_t)m[i] * m[i] * 8);
    P.off_Rtmp = take((size_t)m[i] * m[i] * 8);
    P.off_SS = take((size_t)m[i] * m[i] * 8);
    P.off_TriT = take((size_t)P.mp * P.mp * es);
    P.a_begin = a;
    a += (int64_t)m[i] * v.N1;
    P.b_begin = bb;
    bb += (int64_t)m[i] * p;
    for (int r = 0; r < 3; ++r) {
      P.s_begin[r] = sblk[r];
      sblk[r] += ceil_div(n[i], 32 << r);
    }
    b->maxN2 = std::max(b->maxN2, v.N2);
    b->minN2 = std::min(b->minN2, v.N2);
    b->maxmp = std::max(b->maxmp, P.mp);
  }
  b->itemsA = a;
  b->itemsB = bb;
  for (int r = 0; r < 3; ++r) b->itemsS[r] = sblk[r];
  b->ws_bytes = off + 256;
  const size_t smemA = (size_t)b->maxN2 * es, smemS32 = (size_t)b->maxmp * 32 * es;
  rhqr_status rs = wt == RHQR_F64 ? batch_set_smem<double>(smemA, smemS32) : batch_set_smem<float>(smemA, smemS32);
  if (rs != RHQR_OK) {
    delete b;
    return rs;
  }
  if (cudaMalloc((void **)&b->dev, sizeof(BatchProb) * count) != cudaSuccess) {
    (void)cudaGetLastError();
    delete b;
    return RHQR_ENOMEM;
  }
  if (cudaMemcpy(b->dev, b->host.data(), sizeof(BatchProb) * count, cudaMemcpyHostToDevice) != cudaSuccess) {
    (void)cudaGetLastError();
    cudaFree(b->dev);
    delete b;
    return RHQR_ECUDA;
  }
  *out = b;
  return RHQR_OK;
}

rhqr_status rhqr_batch_workspace_size(rhqr_batch b, size_t *bytes) {
  if (b == nullptr || bytes == nullptr) return RHQR_EINVAL;
  *bytes = b->ws_bytes;
  return RHQR_OK;
}

rhqr_status rhqr_batch_destroy(rhqr_batch b) {
  if (b == nullptr) return RHQR_OK;
  cudaError_t e = cudaFree(b->dev);
  delete b;
  return e == cudaSuccess ? RHQR_OK : RHQR_ECUDA;
}

rhqr_status rhqr_factor_batched(rhqr_batch b, void *ws, size_t ws_bytes, rhqr_info *info, rhqr_stream_t stream) {
  if (b == nullptr || info == nullptr) return RHQR_EINVAL;
  if (ws == nullptr || ws_bytes < b->ws_bytes) return RHQR_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  return b->wt == RHQR_F64 ? batch_run<double>(b, (char *)ws, info, st) : batch_run<float>(b, (char *)ws, info, st);
}

rhqr_status rhqr_batch_tune(rhqr_batch b, void *ws, size_t ws_bytes, rhqr_info *info, int32_t reps,
                            int32_t *choice, rhqr_stream_t stream) {
  if (b == nullptr || info == nullptr || reps < 1 || reps > 1000) return RHQR_EINVAL;
  if (ws == nullptr || ws_bytes < b->ws_bytes) return RHQR_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  rhqr_status r = b->wt == RHQR_F64 ? batch_tune<double>(b, (char *)ws, info, reps, st)
                                    : batch_tune<float>(b, (char *)ws, info, reps, st);
  if (r == RHQR_OK && choice != nullptr) {
    choice[0] = b->a_threads;
    choice[1] = b->solve_rb;
    choice[2] = b->solve_cap;
  }
  return r;
}

rhqr_status rhqr_batch_get_tuning(rhqr_batch b, int32_t *choice) {
  if (b == nullptr || choice == nullptr) return RHQR_EINVAL;
  choice[0] = b->a_threads;
  choice[1] = b->solve_rb;
  choice[2] = b->solve_cap;
  return RHQR_OK;
}

rhqr_status rhqr_batch_set_tuning(rhqr_batch b, const int32_t *choice) {
  if (b == nullptr || choice == nullptr) return RHQR_EINVAL;
  const bool okA = std::find(std::begin(kAThreads), std::end(kAThreads), choice[0]) != std::end(kAThreads);
  const bool okR = std::find(std::begin(kSolveRB), std::end(kSolveRB), choice[1]) != std::end(kSolveRB);
  const bool okC = std::find(std::begin(kSolveCap), std::end(kSolveCap), choice[2]) != std::end(kSolveCap);
  if (!okA || !okR || !okC) return RHQR_EINVAL;
  b->a_threads = choice[0];
  b->solve_rb = choice[1];
  b->solve_cap = choice[2];
  return RHQR_OK;
}

}  // extern "C"
