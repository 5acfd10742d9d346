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
#include "tcgen05.cuh"

namespace rhqr {
namespace stc {
using namespace tc;

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
  rhqr_info *info;
  long long budget;
};

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
  int *err_s = reinterpret_cast<int *>(bars + 5);
  uint64_t *mma_done = bars + 6;

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
    mbar_init(mma_done, 1);
    *abort_s = 0;
    *err_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  fence_before();
  __syncthreads();
  fence_after();
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
          if (!mbar_wait(y_ready, ny & 1u, P.budget, err_s, abort_s)) { ok = false; break; }
          ++ny;
          if (!mbar_wait(d_free, (nd & 1u) ^ 1u, P.budget, err_s, abort_s)) { ok = false; break; }
          fence_after();
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
      mma_quiesce(mma_done);  // no MMA in flight when tensor memory is released
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
          if (!warp_wait(d_ready, nd & 1u, P.budget, err_s, abort_s)) { ok = false; break; }
          fence_after();
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            uint32_t d[32];
            tmem_ld32(tmem + lane_base + (uint32_t)(DCOL + h * 32), d);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 32; ++j) v[h * 32 + j] -= __uint_as_float(d[j]);
          }
          fence_before();
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
          fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(y_ready);
          ++ny;
        }
      }
    }
    (void)ny;
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, 512);
  }
  if (threadIdx.x == 0 && *err_s) set_status(P.info, RHQR_ETIMEOUT, -1);
}

}  // namespace stc

bool solve_tc_supported(int32_t m) { return m >= 1 && m <= stc::MAXP * stc::PW; }

rhqr_status rows_solve_tc(const float *X, int64_t ldx, int64_t row_begin, int64_t nrows, int32_t m,
                          const float *TriT, int32_t mp_tri, float *Y, int64_t ldy, rhqr_info *info, long long budget,
                          cudaStream_t st) {
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
  P.info = info;
  P.budget = budget > 0 ? budget : kDefaultWaitBudget;
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
  const size_t smem = 1024 + stc::OFFDIAG_BYTES + stc::DIAG_BYTES + stc::RDIAG_BYTES + 256;
  RHQR_CUDA_TRY(cudaFuncSetAttribute(stc::solve_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  stc::solve_tc_kernel<<<grid, stc::NUM_THREADS, smem, st>>>(P);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

}  // namespace rhqr
