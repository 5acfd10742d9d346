// Counter-based random operators of the sketches (Section 2.3 leaves the
// generator open; the scheme is fixed by this library):
//   hash(seed, stream, i) = SplitMix64 output function of
//                           (seed * 0x9E3779B97F4A7C15 + stream * 2^56 + i) mod 2^64
//   SRHT signs   (stream 1): D_i = -1 iff the top bit of the hash is set
//   SRHT rows    (stream 2): the k indices with the smallest hash, in increasing order
//   Gaussian     (streams 3, 4; counter r*n + c): Box-Muller with ln and cos summed
//                from their atanh / Taylor series using only correctly rounded
//                add, mul, div and sqrt (no contraction into fused multiply-adds),
//                so every IEEE machine evaluating the same expression gets the
//                same bits.
#include "common.cuh"
#include "rng.cuh"

namespace rhqr {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t stream_base(uint64_t seed, uint32_t stream) {
  return seed * 0x9E3779B97F4A7C15ull + ((uint64_t)stream << 56);
}

// ---------------------------------------------------------------------------
// series coefficients: 1/(2i+1), i < 12, and 1/n! by f[n] = f[n-1] / n, n < 20
// ---------------------------------------------------------------------------
constexpr int kAtanhTerms = 12;
constexpr int kTrigTerms = 10;
constexpr int kCoefCount = kAtanhTerms + 2 * kTrigTerms;

__global__ void series_coefficients_kernel(double *coef) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < kAtanhTerms; ++i) coef[i] = __ddiv_rn(1.0, (double)(2 * i + 1));
  double *f = coef + kAtanhTerms;
  f[0] = 1.0;
  for (int n = 1; n < 2 * kTrigTerms; ++n) f[n] = __ddiv_rn(f[n - 1], (double)n);
}

__device__ __forceinline__ double series_log(double x, const double *inv_odd) {
  const double kLn2 = 0.6931471805599453;
  uint64_t bits = (uint64_t)__double_as_longlong(x);
  int e = (int)((bits >> 52) & 0x7FF) - 1022;
  double f = __longlong_as_double((long long)((bits & 0x000FFFFFFFFFFFFFull) | 0x3FE0000000000000ull));
  if (f < 0.7071067811865476) {
    f = __dmul_rn(f, 2.0);
    e -= 1;
  }
  double s = __ddiv_rn(__dadd_rn(f, -1.0), __dadd_rn(f, 1.0));
  double s2 = __dmul_rn(s, s);
  double p = inv_odd[kAtanhTerms - 1];
  for (int i = kAtanhTerms - 2; i >= 0; --i) p = __dadd_rn(__dmul_rn(p, s2), inv_odd[i]);
  return __dadd_rn(__dmul_rn((double)e, kLn2), __dmul_rn(2.0, __dmul_rn(s, p)));
}

// cos(2 pi t), t in [0, 1): quarter-turn reduction (exact), then the sine or
// cosine Taylor series on [0, pi/4].
__device__ __forceinline__ double series_cos_turns(double t, const double *inv_fact) {
  const double kHalfPi = 1.5707963267948966;
  double t4 = __dmul_rn(4.0, t);
  double q = floor(t4);
  double r = __dadd_rn(t4, -q);
  bool flip = r > 0.5;
  double rr = flip ? __dadd_rn(1.0, -r) : r;
  double y = __dmul_rn(kHalfPi, rr);
  double y2 = __dmul_rn(y, y);
  int qi = (int)q;
  bool want_sin = ((qi & 1) != 0) != flip;
  double v;
  if (want_sin) {
    double p = -inv_fact[2 * kTrigTerms - 1];
    for (int kk = kTrigTerms - 2; kk >= 0; --kk) {
      double c = (kk & 1) ? -inv_fact[2 * kk + 1] : inv_fact[2 * kk + 1];
      p = __dadd_rn(__dmul_rn(p, y2), c);
    }
    v = __dmul_rn(y, p);
  } else {
    double p = -inv_fact[2 * (kTrigTerms - 1)];
    for (int kk = kTrigTerms - 2; kk >= 0; --kk) {
      double c = (kk & 1) ? -inv_fact[2 * kk] : inv_fact[2 * kk];
      p = __dadd_rn(__dmul_rn(p, y2), c);
    }
    v = p;
  }
  return (qi == 1 || qi == 2) ? -v : v;
}

template <class T>
__device__ __forceinline__ T store_gauss(double g);
template <>
__device__ __forceinline__ double store_gauss<double>(double g) { return g; }
template <>
__device__ __forceinline__ float store_gauss<float>(double g) { return __double2float_rn(g); }
template <>
__device__ __forceinline__ __nv_bfloat16 store_gauss<__nv_bfloat16>(double g) {
  return __float2bfloat16_rn(__double2float_rn(g));
}
template <>
__device__ __forceinline__ __half store_gauss<__half>(double g) {
  return __float2half_rn(__double2float_rn(g));
}

// G[r * ldg + c] for r < k, c < n; counter r * n + c.
template <class T>
__global__ void gaussian_kernel(T *G, int64_t ldg, int64_t n, int32_t k, uint64_t base3, uint64_t base4,
                                const double *coef) {
  __shared__ double c_s[kCoefCount];
  if (threadIdx.x < kCoefCount) c_s[threadIdx.x] = coef[threadIdx.x];
  __syncthreads();
  const double *inv_odd = c_s;
  const double *inv_fact = c_s + kAtanhTerms;
  int64_t total = (int64_t)k * n;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = idx / n, c = idx - r * n;
    uint64_t ctr = (uint64_t)idx;
    uint64_t h1 = mix64(base3 + ctr), h2 = mix64(base4 + ctr);
    double u1 = __dmul_rn((double)((h1 >> 11) + 1ull), 0x1p-53);
    double u2 = __dmul_rn((double)(h2 >> 11), 0x1p-53);
    double rad = __dsqrt_rn(__dmul_rn(-2.0, series_log(u1, inv_odd)));
    double g = __dmul_rn(rad, series_cos_turns(u2, inv_fact));
    G[r * ldg + c] = store_gauss<T>(g);
  }
}

// sign bits: word w holds D_{32w..32w+31}, bit set <=> D_i = -1
__global__ void sign_bits_kernel(uint32_t *bits, int64_t N, uint64_t base1) {
  int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t words = (N + 31) / 32;
  if (w >= words) return;
  uint32_t v = 0;
  for (int b = 0; b < 32; ++b) {
    int64_t i = w * 32 + b;
    if (i < N && (mix64(base1 + (uint64_t)i) >> 63)) v |= 1u << b;
  }
  bits[w] = v;
}

__global__ void signs_to_int8_kernel(const uint32_t *bits, int8_t *out, int64_t N) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) out[i] = ((bits[i >> 5] >> (i & 31)) & 1u) ? (int8_t)-1 : (int8_t)1;
}

// ---------------------------------------------------------------------------
// k smallest keys: radix select over 8 passes of 8-bit digits, then an
// order-preserving compaction of {i : key_i <= kth key}.  Keys are distinct
// (SplitMix64's output function is a bijection), so exactly k are selected.
// ---------------------------------------------------------------------------
struct SelectState {
  unsigned long long prefix;
  unsigned int remaining;
  unsigned int pad;
};

__global__ void select_hist_kernel(unsigned int *hist, const SelectState *st, int64_t N, uint64_t base2,
                                   int pass) {
  __shared__ unsigned int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  int shift = 56 - 8 * pass;
  unsigned long long prefix = st->prefix;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = mix64(base2 + (uint64_t)i);
    if (pass == 0 || (key >> (shift + 8)) == prefix) atomicAdd(&h[(key >> shift) & 0xFF], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

__global__ void select_scan_kernel(unsigned int *hist, SelectState *st) {
  if (threadIdx.x == 0) {
    unsigned int rem = st->remaining, cum = 0;
    int d = 0;
    for (; d < 256; ++d) {
      if (cum + hist[d] >= rem) break;
      cum += hist[d];
    }
    if (d > 255) d = 255;  // cannot happen for distinct keys and rem <= count
    st->remaining = rem - cum;
    st->prefix = (st->prefix << 8) | (unsigned long long)d;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
}

constexpr int kCompactBlock = 1024;

__global__ void compact_count_kernel(unsigned int *counts, const SelectState *st, int64_t N, uint64_t base2) {
  int64_t i = (int64_t)blockIdx.x * kCompactBlock + threadIdx.x;
  uint64_t kth = st->prefix;
  int flag = (i < N) && (mix64(base2 + (uint64_t)i) <= kth);
  int c = __syncthreads_count(flag);
  if (threadIdx.x == 0) counts[blockIdx.x] = (unsigned int)c;
}

// exclusive scan of `nb` counts in one block (sequential over chunks of 1024)
__global__ void compact_scan_kernel(unsigned int *counts, int64_t nb) {
  __shared__ unsigned int buf[kCompactBlock];
  __shared__ unsigned int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += kCompactBlock) {
    int64_t i = base + threadIdx.x;
    unsigned int v = (i < nb) ? counts[i] : 0u;
    buf[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < kCompactBlock; off <<= 1) {
      unsigned int t = (threadIdx.x >= (unsigned)off) ? buf[threadIdx.x - off] : 0u;
      __syncthreads();
      buf[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nb) counts[i] = carry + buf[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == kCompactBlock - 1) carry += buf[threadIdx.x];
    __syncthreads();
  }
}

__global__ void compact_write_kernel(int32_t *rows, const unsigned int *offsets, const SelectState *st, int64_t N,
                                     uint64_t base2, int32_t k) {
  __shared__ unsigned int warp_tot[kCompactBlock / 32];
  int64_t i = (int64_t)blockIdx.x * kCompactBlock + threadIdx.x;
  uint64_t kth = st->prefix;
  int flag = (i < N) && (mix64(base2 + (uint64_t)i) <= kth);
  unsigned int ballot = __ballot_sync(0xffffffffu, flag);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned int before = __popc(ballot & ((1u << lane) - 1u));
  if (lane == 0) warp_tot[wid] = __popc(ballot);
  __syncthreads();
  unsigned int woff = 0;
  for (int w = 0; w < wid; ++w) woff += warp_tot[w];
  if (flag) {
    unsigned int pos = offsets[blockIdx.x] + woff + before;
    if (pos < (unsigned)k) rows[pos] = (int32_t)i;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

rhqr_status make_srht_operator(int64_t N, int32_t k, uint64_t seed, uint32_t *sign_bits, int32_t *rows,
                               void *scratch, size_t scratch_bytes, cudaStream_t st) {
  // scratch: SelectState + 256 hist + counts
  int64_t nb = ceil_div(N, kCompactBlock);
  size_t need = 256 + 256 * sizeof(unsigned int) + (size_t)nb * sizeof(unsigned int) + 256;
  if (scratch_bytes < need) return RHQR_ENOMEM;
  char *p = (char *)scratch;
  SelectState *state = (SelectState *)p;
  unsigned int *hist = (unsigned int *)(p + 256);
  unsigned int *counts = (unsigned int *)(p + 256 + 256 * sizeof(unsigned int));
  uint64_t b1 = stream_base(seed, 1), b2 = stream_base(seed, 2);

  int64_t words = ceil_div(N, 32);
  sign_bits_kernel<<<(unsigned)ceil_div(words, 256), 256, 0, st>>>(sign_bits, N, b1);
  RHQR_LAUNCH_CHECK();

  SelectState init{0ull, (unsigned)k, 0u};
  RHQR_CUDA_TRY(cudaMemcpyAsync(state, &init, sizeof(init), cudaMemcpyHostToDevice, st));
  RHQR_CUDA_TRY(cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned int), st));
  unsigned grid = (unsigned)std::min<int64_t>(ceil_div(N, 256), 4096);
  for (int pass = 0; pass < 8; ++pass) {
    select_hist_kernel<<<grid, 256, 0, st>>>(hist, state, N, b2, pass);
    RHQR_LAUNCH_CHECK();
    select_scan_kernel<<<1, 256, 0, st>>>(hist, state);
    RHQR_LAUNCH_CHECK();
  }
  compact_count_kernel<<<(unsigned)nb, kCompactBlock, 0, st>>>(counts, state, N, b2);
  RHQR_LAUNCH_CHECK();
  compact_scan_kernel<<<1, kCompactBlock, 0, st>>>(counts, nb);
  RHQR_LAUNCH_CHECK();
  compact_write_kernel<<<(unsigned)nb, kCompactBlock, 0, st>>>(rows, counts, state, N, b2, k);
  RHQR_LAUNCH_CHECK();
  // cudaMemcpyAsync from a stack variable: wait before returning
  RHQR_CUDA_TRY(cudaStreamSynchronize(st));
  return RHQR_OK;
}

rhqr_status make_gaussian_operator(int64_t n, int32_t k, uint64_t seed, int32_t dtype, void *G, int64_t ldg,
                                   double *coef_scratch, cudaStream_t st) {
  series_coefficients_kernel<<<1, 32, 0, st>>>(coef_scratch);
  RHQR_LAUNCH_CHECK();
  uint64_t b3 = stream_base(seed, 3), b4 = stream_base(seed, 4);
  int64_t total = (int64_t)k * n;
  unsigned grid = (unsigned)std::min<int64_t>(ceil_div(total, 256), 152 * 64);
  switch (dtype) {
    case RHQR_F64:
      gaussian_kernel<double><<<grid, 256, 0, st>>>((double *)G, ldg, n, k, b3, b4, coef_scratch);
      break;
    case RHQR_F32:
      gaussian_kernel<float><<<grid, 256, 0, st>>>((float *)G, ldg, n, k, b3, b4, coef_scratch);
      break;
    case RHQR_BF16:
      gaussian_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>((__nv_bfloat16 *)G, ldg, n, k, b3, b4, coef_scratch);
      break;
    case RHQR_F16:
      gaussian_kernel<__half><<<grid, 256, 0, st>>>((__half *)G, ldg, n, k, b3, b4, coef_scratch);
      break;
    default:
      return RHQR_EINVAL;
  }
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

rhqr_status export_signs(const uint32_t *bits, int8_t *out, int64_t N, cudaStream_t st) {
  signs_to_int8_kernel<<<(unsigned)ceil_div(N, 256), 256, 0, st>>>(bits, out, N);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

}  // namespace rhqr
