// Row-wise triangular solve Y = X Tri^{-1} (Tri upper triangular, m <= 256)
// for float32 data on the tcgen05 tensor cores.  With Tri = R this forms the
// recRHQR factor Q = W R^{-1} (Section 3.3).
//
// Columns are processed in panels of 64, left-looking, for tiles of 128 rows:
//   D_J   = sum_{I < J} Y_I Tri_{I,J}                (tensor cores)
//   Y_J   = (X_J - D_J) Tri_{J,J}^{-1}              (forward substitution in
//                                                     float32, one thread per row)
// so every row is still solved by a backward-stable substitution; only the
// off-diagonal products go through the tensor cores, with both operands split
// exactly into three bf16 limbs (float32 values are sums of three bf16
// numbers).  The six limb products with weight >= 2^-16 are issued smallest
// first, so the float32 accumulator's per-MMA truncation only acts at the
// magnitude of the final sum.
//
// Operands: Y limbs live in tensor memory (the A operand of kind::f16 may be
// read from tensor memory: row i in lane i, two bf16 per 32-bit column); the
// off-diagonal blocks of Tri (as B = N x K, K-major, 128-byte swizzle) and
// the float32 diagonal blocks live in shared memory for the whole persistent
// CTA.  Tensor memory: 3 limbs x 4 panels x 32 columns of Y + 64 columns of D.
//
// Roles: warp 1 allocates tensor memory and issues the MMAs; warps 4..7 (one
// thread per tile row) load X, finish each panel, store Q and write the Y
// limbs.  All mbarrier waits are bounded.
#include "solve_tc.cuh"

namespace rhqr {
namespace stc {

constexpr int TILE = 128;
constexpr int PW = 64;    // panel width
constexpr int MAXP = 4;   // panels (m <= 256)
constexpr int NUM_THREADS = 256;
constexpr int SOLVE_WARP0 = 4;
constexpr int BLK_BYTES = PW * PW * 2;        // one bf16 limb of a 64 x 64 block: 8 KiB
constexpr int OFFDIAG_BYTES = 6 * 3 * BLK_BYTES;  // 6 blocks x 3 limbs: 144 KiB
constexpr int DIAG_BYTES = MAXP * PW * PW * 4;    // 64 KiB
constexpr int RDIAG_BYTES = MAXP * PW * 4;        // reciprocals of the diagonal
constexpr int YCOL = 0;     // tensor-memory column of the Y limbs
constexpr int DCOL = 384;   // tensor-memory column of D

struct Params {
  const float *X;
  int64_t ldx;
  float *Y;
  int64_t ldy;
  int64_t row_begin, nrows;
  int32_t m, P;        // columns, panels (P = ceil(m / 64))
  const float *TriT;   // mp x mp row-major: TriT[l * mp + j] = Tri[l, j], identity-padded
  int32_t mp;
  int *err;
  long long budget;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long budget, int *err,
                                          volatile int *abort_s) {
  long long it = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_s) return false;
    if (++it > budget) {
      atomicExch(err, 1);
      *abort_s = 1;
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, long long budget, int *err,
                                          volatile int *abort_s) {
  bool ok = mbar_wait(bar, parity, budget, err, abort_s);
  return __all_sync(0xffffffffu, ok);
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// D[tmem] (+)= A[tmem] * B[smem]^T, kind::f16, bf16 inputs, f32 accumulate
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

#define STC_R32(r)                                                                                               \
  "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),    \
      "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),     \
      "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),    \
      "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
#define STC_W32(r)                                                                                                \
  "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),   \
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), \
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), \
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : STC_R32(r)
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      STC_W32(r)
      : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// index of the off-diagonal block (I, J), I < J < 4, in 0..5
__host__ __device__ constexpr int blk_index(int I, int J) { return J * (J - 1) / 2 + I; }

__device__ __forceinline__ void split3(float x, __nv_bfloat16 &h, __nv_bfloat16 &mi, __nv_bfloat16 &lo) {
  h = __float2bfloat16_rn(x);
  float r1 = x - __bfloat162float(h);
  mi = __float2bfloat16_rn(r1);
  float r2 = r1 - __bfloat162float(mi);
  lo = __float2bfloat16_rn(r2);
}

__global__ void __launch_bounds__(NUM_THREADS, 1) solve_tc_kernel(Params P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *offdiag = smem;                                      // 6 blocks x 3 limbs
  float *diag = reinterpret_cast<float *>(smem + OFFDIAG_BYTES);  // 4 x 64 x 64, row-major
  float *rdiag = reinterpret_cast<float *>(smem + OFFDIAG_BYTES + DIAG_BYTES);
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + OFFDIAG_BYTES + DIAG_BYTES + RDIAG_BYTES);
  uint64_t *y_ready = bars, *d_ready = bars + 1, *d_free = bars + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 3);
  volatile int *abort_s = reinterpret_cast<volatile int *>(bars + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NP = P.P, mp = P.mp;

  // ---- stage Tri in shared memory: diagonal blocks (float32) and the
  //      off-diagonal blocks as B operands (N = 64 columns x K = 64 rows)
  for (int e = threadIdx.x; e < NP * PW * PW; e += NUM_THREADS) {
    int J = e / (PW * PW), rr = (e / PW) % PW, cc = e % PW;
    diag[e] = P.TriT[(int64_t)(J * PW + rr) * mp + J * PW + cc];
  }
  for (int e = threadIdx.x; e < NP * PW; e += NUM_THREADS) {
    const int J = e / PW, d = e % PW;
    rdiag[e] = __frcp_rn(P.TriT[(int64_t)(J * PW + d) * mp + J * PW + d]);
  }
  for (int J = 1; J < NP; ++J)
    for (int I = 0; I < J; ++I) {
      uint8_t *blk = offdiag + (size_t)blk_index(I, J) * 3 * BLK_BYTES;
      // B row n = column J*64+n of Tri; 8 chunks of 8 K-values (rows I*64 + 8*c .. +7)
      for (int q = threadIdx.x; q < PW * 8; q += NUM_THREADS) {
        int nrow = q >> 3, chunk = q & 7;
        uint32_t w[3][4];
#pragma unroll
        for (int e2 = 0; e2 < 4; ++e2) {
          float a = P.TriT[(int64_t)(I * PW + chunk * 8 + 2 * e2) * mp + J * PW + nrow];
          float b = P.TriT[(int64_t)(I * PW + chunk * 8 + 2 * e2 + 1) * mp + J * PW + nrow];
          __nv_bfloat16 ah, am, al, bh, bm, bl;
          split3(a, ah, am, al);
          split3(b, bh, bm, bl);
          w[0][e2] = (uint32_t)__bfloat16_as_ushort(ah) | ((uint32_t)__bfloat16_as_ushort(bh) << 16);
          w[1][e2] = (uint32_t)__bfloat16_as_ushort(am) | ((uint32_t)__bfloat16_as_ushort(bm) << 16);
          w[2][e2] = (uint32_t)__bfloat16_as_ushort(al) | ((uint32_t)__bfloat16_as_ushort(bl) << 16);
        }
        const uint32_t off = (uint32_t)nrow * 128u + ((uint32_t)(chunk ^ (nrow & 7)) << 4);
#pragma unroll
        for (int l = 0; l < 3; ++l)
          *reinterpret_cast<uint4 *>(blk + l * BLK_BYTES + off) = make_uint4(w[l][0], w[l][1], w[l][2], w[l][3]);
      }
    }
  fence_proxy_async();
  if (threadIdx.x == 0) {
    mbar_init(y_ready, 4);
    mbar_init(d_ready, 1);
    mbar_init(d_free, 4);
    *abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t ntiles = (P.nrows + TILE - 1) / TILE;
  if (warp == 1) {
    if (lane == 0 && NP > 1) {
      const uint32_t idesc = idesc_bf16(128, PW);
      // limb products (a of Y, b of Tri) with weight >= 2^-16, smallest first
      const int pa[6] = {2, 1, 0, 1, 0, 0};
      const int pb[6] = {0, 1, 2, 0, 1, 0};
      uint32_t ny = 0, nd = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        for (int J = 1; J < NP; ++J) {
          if (!mbar_wait(y_ready, ny & 1u, P.budget, P.err, abort_s)) { ok = false; break; }
          ++ny;
          if (!mbar_wait(d_free, (nd & 1u) ^ 1u, P.budget, P.err, abort_s)) { ok = false; break; }
          tc_fence_after();
          int first = 1;
          for (int pr = 0; pr < 6; ++pr)
            for (int I = 0; I < J; ++I)
              for (int kk = 0; kk < PW / 16; ++kk) {
                const uint32_t a_t = tmem + (uint32_t)(YCOL + (pa[pr] * MAXP + I) * 32 + kk * 8);
                const uint32_t b_s = smem_u32(offdiag + (size_t)blk_index(I, J) * 3 * BLK_BYTES +
                                              (size_t)pb[pr] * BLK_BYTES) + kk * 32;
                mma_ts(tmem + DCOL, a_t, sw128_desc(b_s), idesc, first ? 0u : 1u);
                first = 0;
              }
          mma_commit(d_ready);
          ++nd;
        }
      }
    }
  } else if (warp >= SOLVE_WARP0) {
    const int qd = warp & 3;
    const int r = qd * 32 + lane;
    const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
    uint32_t ny = 0, nd = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const int64_t row = P.row_begin + t * TILE + r;
      const bool live = (t * TILE + r) < P.nrows;
      for (int J = 0; J < NP; ++J) {
        float v[PW];
#pragma unroll
        for (int c = 0; c < PW; ++c) {
          const int col = J * PW + c;
          v[c] = (live && col < P.m) ? __ldg(P.X + (int64_t)col * P.ldx + row) : 0.f;
        }
        if (J > 0) {
          if (!warp_wait(d_ready, nd & 1u, P.budget, P.err, abort_s)) { ok = false; break; }
          tc_fence_after();
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            uint32_t d[32];
            tmem_ld32(tmem + lane_base + (uint32_t)(DCOL + h * 32), d);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 32; ++j) v[h * 32 + j] -= __uint_as_float(d[j]);
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(d_free);
          ++nd;
        }
        // forward substitution with the diagonal block (row-major, upper)
        const float *dg = diag + J * PW * PW;
#pragma unroll
        for (int jj = 0; jj < PW; ++jj) {
          v[jj] *= rdiag[J * PW + jj];
#pragma unroll
          for (int q4 = ((jj + 1) & ~3); q4 < PW; q4 += 4) {
            const float4 rr = *reinterpret_cast<const float4 *>(dg + jj * PW + q4);
            if (q4 + 0 > jj) v[q4 + 0] -= v[jj] * rr.x;
            if (q4 + 1 > jj) v[q4 + 1] -= v[jj] * rr.y;
            if (q4 + 2 > jj) v[q4 + 2] -= v[jj] * rr.z;
            if (q4 + 3 > jj) v[q4 + 3] -= v[jj] * rr.w;
          }
        }
        if (live) {
#pragma unroll
          for (int c = 0; c < PW; ++c) {
            const int col = J * PW + c;
            if (col < P.m) P.Y[(int64_t)col * P.ldy + row] = v[c];
          }
        }
        if (J < NP - 1) {
          // three bf16 limbs of Y_J into tensor memory (two values per column),
          // 16 columns (32 values) at a time
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            uint32_t w0[16], w1[16], w2[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              __nv_bfloat16 ah, am, al, bh, bm, bl;
              split3(v[32 * h + 2 * j], ah, am, al);
              split3(v[32 * h + 2 * j + 1], bh, bm, bl);
              w0[j] = (uint32_t)__bfloat16_as_ushort(ah) | ((uint32_t)__bfloat16_as_ushort(bh) << 16);
              w1[j] = (uint32_t)__bfloat16_as_ushort(am) | ((uint32_t)__bfloat16_as_ushort(bm) << 16);
              w2[j] = (uint32_t)__bfloat16_as_ushort(al) | ((uint32_t)__bfloat16_as_ushort(bl) << 16);
            }
            const uint32_t col = tmem + lane_base + (uint32_t)(YCOL + J * 32 + h * 16);
            tmem_st16(col + (uint32_t)(0 * MAXP * 32), w0);
            tmem_st16(col + (uint32_t)(1 * MAXP * 32), w1);
            tmem_st16(col + (uint32_t)(2 * MAXP * 32), w2);
          }
          tmem_wait_st();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(y_ready);
          ++ny;
        }
      }
    }
    (void)ny;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

}  // namespace stc

bool solve_tc_supported(int32_t m) { return m >= 1 && m <= stc::MAXP * stc::PW; }

rhqr_status rows_solve_tc(const float *X, int64_t ldx, int64_t row_begin, int64_t nrows, int32_t m,
                          const float *TriT, int32_t mp_tri, float *Y, int64_t ldy, int *err, cudaStream_t st) {
  if (nrows <= 0) return RHQR_OK;
  if (!solve_tc_supported(m)) return RHQR_ENOTSUP;
  stc::Params P;
  P.X = X;
  P.ldx = ldx;
  P.Y = Y;
  P.ldy = ldy;
  P.row_begin = row_begin;
  P.nrows = nrows;
  P.m = m;
  P.P = (int32_t)ceil_div(m, stc::PW);
  P.TriT = TriT;
  P.mp = mp_tri;
  P.err = err;
  P.budget = 4000000LL;
  if (P.mp < P.P * stc::PW) return RHQR_EINVAL;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  const int64_t ntiles = ceil_div(nrows, stc::TILE);
  const unsigned grid = (unsigned)std::min<int64_t>(ntiles, sms);
  const size_t smem = 1024 + stc::OFFDIAG_BYTES + stc::DIAG_BYTES + stc::RDIAG_BYTES + 128;
  RHQR_CUDA_TRY(cudaFuncSetAttribute(stc::solve_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  RHQR_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  stc::solve_tc_kernel<<<grid, stc::NUM_THREADS, smem, st>>>(P);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

}  // namespace rhqr
