// Gaussian sketch Omega X on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Z_Omega = G X_2 / sqrt(k) (Section 2.3) with G (k x n) stored in bf16 or f16
// and X (n x c) in float32.  X is split into L 16-bit limbs,
// X = X_1 + ... + X_L (X_1 = round(X), X_2 = round(X - X_1), ...), so that the
// products of the stored G with every limb are exact.
//
// Tensor-core accumulation adds each 16-deep product block to the float32
// accumulator with truncation, so its error grows with the number of MMAs
// that hit one accumulator.  The accumulator is therefore drained every
// `kdrain` rows of X into a float32 running sum kept in the other half of
// tensor memory and updated with round-to-nearest adds; the per-chunk results
// are summed in float64 in a fixed order.
//
// One CTA owns a 256 x Nt output tile (Nt <= 128 columns) and one K-chunk of
// X rows.  The tile is accumulated transposed: tensor-memory lane = column of
// X (the limbs are the M = 128 operand), accumulator column = row of G (the G
// tile is the N = 256 operand), so one MMA per 16 rows and limb reads G once
// for both halves of the tile and the accumulator takes 256 of the 512
// tensor-memory columns, leaving the other 256 for the running sum.
//   warp 0       : producer: per stage the G tile (256 x 64, one contiguous
//                  32 KiB bulk copy from the operator's tile-order copy, which
//                  holds it already in the 128-byte swizzled layout) and the
//                  X tile (64 rows x Nt float32, TMA)
//   warp 1       : tensor-memory allocation and the single MMA-issuing thread
//   warps 2..7   : converters: staged X -> L limbs in the K-major 128-byte
//                  swizzled layout the MMA reads (rows < m are zeroed)
//   warps 8..15  : drainers: fresh accumulator + running sum -> running sum;
//                  at the end the running sums go to a float32 partial
//                  [chunk][row][column] in global memory
// Every wait on an mbarrier is bounded; a wait that runs out sets an error
// flag, the other roles stop, TMA copies still in flight are awaited (bounded)
// and tensor memory is released before the block exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "sketch_tc.cuh"
#include "tcgen05.cuh"
#include "tma_host.cuh"

namespace rhqr {
namespace tc {

constexpr int BM = 256;  // rows of G per CTA
constexpr int BK = 64;   // rows of X per stage (128 bytes of a 16-bit limb)
constexpr int NT = 128;  // max columns of X per CTA
constexpr int MAXC = 256;
constexpr int NUM_THREADS = 512;
constexpr int CONV_WARP0 = 2, NUM_CONV_WARPS = 6;
constexpr int DRAIN_WARP0 = 8, NUM_DRAIN_WARPS = 8;
constexpr int A_BYTES = BM * BK * 2;    // 32 KiB
constexpr int B_BYTES = NT * BK * 2;    // 16 KiB per limb
constexpr int X_BYTES = NT * BK * 4;    // 32 KiB staging
constexpr int KDRAIN = 256;             // rows of X between drains
constexpr int RUN_COL = 256;            // tensor-memory column of the running sums

struct Params {
  int64_t n;
  int32_t m, m64, c, Nt, k;
  int64_t kchunk;
  int32_t limbs, stages, kdrain;
  int32_t xbytes;  // bytes of one X box: 64 rows x Nt columns of float32
  float *part;  // [nch][k][c]
  const char *gt;  // operator tiles (256 x 64, 32 KiB each), gt_nkb per row of tiles
  int64_t gt_nkb;
  const float *colscale;  // per column of X: exact power-of-two scale before the limb split, or NULL
  int *err;
  long long budget;
};

template <class TL>
struct Limb;
template <>
struct Limb<__nv_bfloat16> {
  static constexpr uint32_t fmt = 1;
  __device__ static __forceinline__ uint32_t pack(float a, float b, float &ra, float &rb) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // one packed conversion: a low, b high
    const float2 hf = __bfloat1622float2(h);
    ra = a - hf.x;
    rb = b - hf.y;
    return *reinterpret_cast<const uint32_t *>(&h);
  }
};
template <>
struct Limb<__half> {
  static constexpr uint32_t fmt = 0;
  __device__ static __forceinline__ uint32_t pack(float a, float b, float &ra, float &rb) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    ra = a - hf.x;
    rb = b - hf.y;
    return *reinterpret_cast<const uint32_t *>(&h);
  }
};

// Converters, limbs written in place (L <= 2): one warp per group of 8 columns
// (2 KiB of float32, 64 rows each).  Load e4 of lane l is float4 f = 32 e4 + l:
// column f / 16, rows 4 (f % 16) .. + 3, so each 8-lane phase reads 128
// contiguous bytes (no bank conflicts); the lane then writes its 4 rows of each
// limb as 8 bytes of the swizzled atom row of that column.  Rows below m (the
// exact top block) are zeroed.
template <class TL, int L>
__device__ __forceinline__ void convert_inplace(const float *xs, uint8_t *bst_in, const Params &P, int col0,
                                                int64_t r0, int wg, int lane) {
  const bool top = r0 < P.m;
  for (int g = wg; g < P.Nt / 8; g += NUM_CONV_WARPS) {
    const float4 *src = reinterpret_cast<const float4 *>(xs + 8 * g * BK);
    float v[16];
#pragma unroll
    for (int e4 = 0; e4 < 4; ++e4) {
      const float4 f = src[32 * e4 + lane];
      v[4 * e4] = f.x, v[4 * e4 + 1] = f.y, v[4 * e4 + 2] = f.z, v[4 * e4 + 3] = f.w;
    }
    if (P.colscale != nullptr) {
#pragma unroll
      for (int e4 = 0; e4 < 4; ++e4) {
        const int col = col0 + 8 * g + 2 * e4 + (lane >> 4);
        const float sc = col < P.c ? P.colscale[col] : 1.f;
#pragma unroll
        for (int e = 0; e < 4; ++e) v[4 * e4 + e] *= sc;
      }
    }
    if (top) {
#pragma unroll
      for (int e4 = 0; e4 < 4; ++e4)
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (r0 + 4 * ((32 * e4 + lane) & 15) + e < P.m) v[4 * e4 + e] = 0.f;
    }
    __syncwarp();  // the whole group is read before its bytes are overwritten
    uint8_t *atom = bst_in + g * 2048;
#pragma unroll
    for (int e4 = 0; e4 < 4; ++e4) {
      const int f = 32 * e4 + lane, n = f >> 4, row = 4 * (f & 15);
      const uint32_t off =
          (uint32_t)n * 128u + ((((uint32_t)row >> 3) ^ (uint32_t)(n & 7)) << 4) + (uint32_t)((row & 7) * 2);
      float *vv = v + 4 * e4;
#pragma unroll
      for (int l = 0; l < L; ++l) {
        float rr[4];
        uint2 w;
        w.x = Limb<TL>::pack(vv[0], vv[1], rr[0], rr[1]);
        w.y = Limb<TL>::pack(vv[2], vv[3], rr[2], rr[3]);
        *reinterpret_cast<uint2 *>(atom + l * 1024 + off) = w;
#pragma unroll
        for (int e = 0; e < 4; ++e) vv[e] = rr[e];
      }
    }
    __syncwarp();
  }
}

// Drainers, one drain: thread -> one column of X (tensor-memory lane), 128
// accumulator columns (rows of G) starting at `fresh`; the running sums at
// `run` take the fresh accumulator with round-to-nearest adds, and the last
// drain writes them to the float32 partial of chunk `ch`.  The warp arrives on
// `release` (the MMAs may overwrite the fresh accumulator) as soon as its last
// load of it has completed, before the last adds and stores of the running sum.
__device__ __forceinline__ void drain_once(uint32_t fresh, uint32_t run, bool first, bool last, bool own_col,
                                           float unscale, int row0, int cc, int ch, const Params &P,
                                           uint64_t *release) {
  for (int c0 = 0; c0 < 128; c0 += 32) {
    uint32_t f[32], r[32];
    tmem_ld32(fresh + c0, f);
    if (!first) tmem_ld32(run + c0, r);
    tmem_wait_ld();
    if (c0 == 96) {
      fence_before();
      __syncwarp();
      if ((threadIdx.x & 31) == 0) mbar_arrive(release);
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      float v = __uint_as_float(f[j]);
      if (!first) v = __fadd_rn(__uint_as_float(r[j]), v);
      r[j] = __float_as_uint(v);
    }
    if (last) {
      if (own_col) {
        for (int j = 0; j < 32; ++j) {
          const int row = row0 + c0 + j;
          if (row < P.k) P.part[((int64_t)ch * P.k + row) * P.c + cc] = __uint_as_float(r[j]) * unscale;
        }
      }
    } else {
      tmem_st32(run + c0, r);
    }
  }
  tmem_wait_st();
}

template <class TL, int L>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    sketch_tc_kernel(const __grid_constant__ CUtensorMap tmapX, Params P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // With up to two limbs, X is split in place: the float32 staging of 8 columns
  // (2 KiB) becomes their limb atoms (8 rows x 128 bytes each, 2 KiB apart per
  // limb pair), so a stage is A | X and three stages fit; three limbs need a
  // separate limb area (A | X staging | limbs, two stages).
  constexpr bool INPLACE = L <= 2;
  const int S = P.stages;
  const int stage_bytes = INPLACE ? A_BYTES + X_BYTES : A_BYTES + X_BYTES + L * B_BYTES;
  uint64_t *bars = (uint64_t *)(smem + S * stage_bytes);
  uint64_t *full_a = bars, *full_b = bars + 4, *empty = bars + 8, *xempty = bars + 12;
  uint64_t *fresh_full = bars + 16, *fresh_empty = bars + 17;
  uint32_t *tmem_slot = (uint32_t *)(bars + 18);
  volatile int *abort_s = (volatile int *)(bars + 19);
  uint64_t *mma_done = bars + 20;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = blockIdx.x, nt = blockIdx.y, ch = blockIdx.z;
  const int col0 = nt * P.Nt;
  // chunks start on 64-row boundaries (whole operator tiles); rows below m
  // (the exact top block) are zeroed by the converters
  const int64_t x_begin = (int64_t)P.m64 + (int64_t)ch * P.kchunk;
  const int64_t x_end = min(P.n, x_begin + P.kchunk);
  const int steps = (int)((x_end - x_begin + BK - 1) / BK);
  const int per_drain = P.kdrain / BK;
  const int drains = (steps + per_drain - 1) / per_drain;

  if (threadIdx.x == 0) {
    for (int s = 0; s < 4; ++s) {
      mbar_init(full_a + s, 1);
      mbar_init(full_b + s, NUM_CONV_WARPS);
      mbar_init(empty + s, 1);
      mbar_init(xempty + s, NUM_CONV_WARPS);
    }
    mbar_init(fresh_full, 1);
    mbar_init(fresh_empty, NUM_DRAIN_WARPS);
    mbar_init(mma_done, 1);
    *abort_s = 0;
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

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < steps; ++i) {
        const int s = i % S;
        const uint32_t ph = (uint32_t)(i / S) & 1u;
        if (!mbar_wait(empty + s, ph ^ 1u, P.budget, P.err, abort_s) ||
            (!INPLACE && !mbar_wait(xempty + s, ph ^ 1u, P.budget, P.err, abort_s)))
          break;
        uint8_t *st = smem + s * stage_bytes;
        mbar_expect_tx(full_a + s, (uint32_t)(A_BYTES + P.xbytes));
        const int xr = (int)(x_begin + (int64_t)i * BK);
        bulk_load(st, P.gt + ((int64_t)mt * P.gt_nkb + xr / BK) * A_BYTES, A_BYTES, full_a + s);
        tma_load_2d(st + A_BYTES, &tmapX, full_a + s, xr, col0);
        ++issued;
      }
      // the last copies issued into each stage complete before the block exits
      // (already so on the normal path; after a stop they may still be in flight)
      for (int i = max(0, issued - S); i < issued; ++i) drain_wait(full_a + (i % S), (uint32_t)(i / S) & 1u);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(128, BM, Limb<TL>::fmt);  // M: 128 columns of X, N: 256 rows of G
      int i = 0;
      for (int d = 0; d < drains && i < steps; ++d) {
        if (d > 0 && !mbar_wait(fresh_empty, (uint32_t)(d - 1) & 1u, P.budget, P.err, abort_s)) break;
        fence_after();
        bool ok = true;
        for (int j = 0; j < per_drain && i < steps; ++j, ++i) {
          const int s = i % S;
          const uint32_t ph = (uint32_t)(i / S) & 1u;
          if (!mbar_wait(full_a + s, ph, P.budget, P.err, abort_s) ||
              !mbar_wait(full_b + s, ph, P.budget, P.err, abort_s)) {
            ok = false;
            break;
          }
          fence_after();
          // descriptors advance by (byte offset >> 4): the loops unroll to constant adds
          const uint32_t st_base = smem_u32(smem + s * stage_bytes);
          const uint64_t gd0 = sw128_desc(st_base);  // G: 256 rows of 128 bytes
          const uint64_t xd0 = INPLACE ? sw128_desc(st_base + A_BYTES, 2048) : sw128_desc(st_base + A_BYTES + X_BYTES);
          constexpr int LIMB_STRIDE = INPLACE ? 1024 : B_BYTES;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
#pragma unroll
            for (int l = 0; l < L; ++l)
              mma_ss(tmem, xd0 + (uint64_t)((l * LIMB_STRIDE + kk * 32) >> 4), gd0 + (uint64_t)((kk * 32) >> 4),
                      idesc, (uint32_t)(j != 0 || kk != 0 || l != 0));
          mma_commit(empty + s);
        }
        mma_commit(fresh_full);
        if (!ok) break;
      }
      mma_quiesce(mma_done);  // no MMA in flight when tensor memory is released
    }
  } else if (warp >= CONV_WARP0 && warp < CONV_WARP0 + NUM_CONV_WARPS) {
    // converters: 128 threads, X staging (col-major 64 rows x Nt) -> limbs
    const int ct = threadIdx.x - CONV_WARP0 * 32;
    for (int i = 0; i < steps; ++i) {
      const int s = i % S;
      const uint32_t ph = (uint32_t)(i / S) & 1u;
      if (!warp_wait(full_a + s, ph, P.budget, P.err, abort_s)) break;
      uint8_t *st = smem + s * stage_bytes;
      const float *xs = reinterpret_cast<const float *>(st + A_BYTES);
      uint8_t *bst = st + A_BYTES + X_BYTES;
      uint8_t *bst_in = st + A_BYTES;
      const int64_t r0 = x_begin + (int64_t)i * BK;
      const bool top = r0 < P.m;  // rows below m are the exact top block: excluded
      if (INPLACE) {
        convert_inplace<TL, L>(xs, bst_in, P, col0, r0, warp - CONV_WARP0, lane);
      } else
      for (int q = ct; q < P.Nt * 8; q += NUM_CONV_WARPS * 32) {
        const int nn = q >> 3, cidx = q & 7;
        const float4 *src = reinterpret_cast<const float4 *>(xs + nn * BK + cidx * 8);
        float4 a = src[0], b = src[1];
        float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        if (P.colscale != nullptr) {
          const float sc = col0 + nn < P.c ? P.colscale[col0 + nn] : 1.f;
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] *= sc;
        }
        if (top) {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (r0 + cidx * 8 + e < P.m) v[e] = 0.f;
        }
        const uint32_t off = (uint32_t)nn * 128u + ((uint32_t)(cidx ^ (nn & 7)) << 4);
#pragma unroll
        for (int l = 0; l < L; ++l) {
          uint4 w;
          float r[8];
          w.x = Limb<TL>::pack(v[0], v[1], r[0], r[1]);
          w.y = Limb<TL>::pack(v[2], v[3], r[2], r[3]);
          w.z = Limb<TL>::pack(v[4], v[5], r[4], r[5]);
          w.w = Limb<TL>::pack(v[6], v[7], r[6], r[7]);
          *reinterpret_cast<uint4 *>(bst + l * B_BYTES + off) = w;
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = r[e];
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(full_b + s);
        mbar_arrive(xempty + s);
      }
    }
  } else if (warp >= DRAIN_WARP0) {
    // drainers: warp -> (half h of the G rows, lane quarter qd); thread -> one
    // column of X (tensor-memory lane), 128 accumulator columns (rows of G)
    const int dw = warp - DRAIN_WARP0;
    const int h = dw >> 2, qd = warp & 3;
    const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
    const uint32_t fresh = tmem + lane_base + (uint32_t)(h * 128);
    const uint32_t run = tmem + lane_base + (uint32_t)(RUN_COL + h * 128);
    const int cc = col0 + qd * 32 + lane;
    const bool own_col = qd * 32 + lane < P.Nt && cc < P.c;
    const float unscale = (own_col && P.colscale != nullptr) ? 1.f / P.colscale[cc] : 1.f;  // a power of two
    const int row0 = mt * BM + h * 128;
    bool ok = true;
    for (int d = 0; d < drains; ++d) {
      if (!warp_wait(fresh_full, (uint32_t)d & 1u, P.budget, P.err, abort_s)) {
        ok = false;
        break;
      }
      fence_after();
      drain_once(fresh, run, d == 0, d == drains - 1, own_col, unscale, row0, cc, ch, P, fresh_empty);
    }
    (void)ok;
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// The same sketch on CTA pairs (cta_group::2), for two column tiles of X
// (128 < c <= 256) and L <= 2 limbs.  The pair (a cluster of 2 along x: rank
// 0 and 1 = column tiles 0 and 1 of one G tile and K-chunk) issues one
// M = 256, N = 256 MMA per 16 rows and limb: M covers the two CTAs' 128
// columns of X each, and the G tile's 256 rows are split between them, rank r
// holding rows 128 r .. 128 r + 127.  Each SM thus stages and reads half of G,
// the operand that dominates the shared-memory reads of the single-CTA
// kernel, while its tensor memory still receives all 256 rows of G for its
// 128 columns.  Rank 0 issues the MMAs once both CTAs' converters have filled
// a stage, and its commits arrive on both CTAs' barriers.  Converters and
// drainers arrive on their own CTA's barriers only (an arrival with
// cluster-scope release costs more than the conversion of a stage); in rank
// 1, two lanes of the otherwise idle warp 1 wait for each completed stage and
// each completed drain and forward it to rank 0 with one remote arrival.
constexpr int G_HALF_BYTES = A_BYTES / 2;  // 128 rows of the G tile
constexpr int PAIR_STAGES = 4;

template <class TL, int L>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    sketch_tc_pair_kernel(const __grid_constant__ CUtensorMap tmapX, Params P) {
  static_assert(L <= 2, "limbs are written in place");
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int S = PAIR_STAGES;
  constexpr int stage_bytes = G_HALF_BYTES + X_BYTES;
  uint64_t *bars = (uint64_t *)(smem + S * stage_bytes);
  uint64_t *full_a = bars, *full_b = bars + S, *empty = bars + 2 * S;
  uint64_t *fresh_full = bars + 3 * S, *fresh_empty = bars + 3 * S + 1, *mma_done = bars + 3 * S + 2;
  uint32_t *tmem_slot = (uint32_t *)(bars + 3 * S + 3);
  volatile int *abort_s = (volatile int *)(bars + 3 * S + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();  // = blockIdx.x: column tile
  const bool leader = rank == 0;
  const int mt = blockIdx.y, ch = blockIdx.z;
  const int col0 = (int)rank * P.Nt;
  const int64_t x_begin = (int64_t)P.m64 + (int64_t)ch * P.kchunk;
  const int64_t x_end = min(P.n, x_begin + P.kchunk);
  const int steps = (int)((x_end - x_begin + BK - 1) / BK);
  const int per_drain = P.kdrain / BK;
  const int drains = (steps + per_drain - 1) / per_drain;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full_a + s, 1);
      mbar_init(full_b + s, leader ? NUM_CONV_WARPS + 1 : NUM_CONV_WARPS);  // rank 0: + rank 1's forward
      mbar_init(empty + s, 1);
    }
    mbar_init(fresh_full, 1);
    mbar_init(fresh_empty, leader ? NUM_DRAIN_WARPS + 1 : NUM_DRAIN_WARPS);
    mbar_init(mma_done, 1);
    *abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc2(tmem_slot, 512);
    tmem_relinquish2();
  }
  fence_before();
  __syncthreads();
  fence_after();
  cluster_sync();  // both CTAs' barriers are initialised before any remote arrival
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // producer (both CTAs): this CTA's half of the G tile and its X tile
      int issued = 0;
      for (int i = 0; i < steps; ++i) {
        const int s = i % S;
        const uint32_t ph = (uint32_t)(i / S) & 1u;
        if (!mbar_wait(empty + s, ph ^ 1u, P.budget, P.err, abort_s)) break;
        uint8_t *st = smem + s * stage_bytes;
        mbar_expect_tx(full_a + s, (uint32_t)(G_HALF_BYTES + P.xbytes));
        const int xr = (int)(x_begin + (int64_t)i * BK);
        bulk_load(st, P.gt + ((int64_t)mt * P.gt_nkb + xr / BK) * A_BYTES + (int64_t)rank * G_HALF_BYTES,
                  G_HALF_BYTES, full_a + s);
        tma_load_2d(st + G_HALF_BYTES, &tmapX, full_a + s, xr, col0);
        ++issued;
      }
      for (int i = max(0, issued - S); i < issued; ++i) drain_wait(full_a + (i % S), (uint32_t)(i / S) & 1u);
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      const uint32_t idesc = idesc_f16(256, BM, Limb<TL>::fmt);  // M: the pair's 256 columns of X, N: 256 rows of G
      int i = 0;
      for (int d = 0; d < drains && i < steps; ++d) {
        if (d > 0 && !mbar_wait_cluster(fresh_empty, (uint32_t)(d - 1) & 1u, P.budget, P.err, abort_s)) break;
        fence_after();
        bool ok = true;
        for (int j = 0; j < per_drain && i < steps; ++j, ++i) {
          const int s = i % S;
          const uint32_t ph = (uint32_t)(i / S) & 1u;
          if (!mbar_wait(full_a + s, ph, P.budget, P.err, abort_s) ||
              !mbar_wait_cluster(full_b + s, ph, P.budget, P.err, abort_s)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t st_base = smem_u32(smem + s * stage_bytes);
          const uint64_t gd0 = sw128_desc(st_base);                       // this CTA's 128 rows of G
          const uint64_t xd0 = sw128_desc(st_base + G_HALF_BYTES, 2048);  // limbs, written in place
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
#pragma unroll
            for (int l = 0; l < L; ++l)
              mma_ss2(tmem, xd0 + (uint64_t)((l * 1024 + kk * 32) >> 4), gd0 + (uint64_t)((kk * 32) >> 4), idesc,
                      (uint32_t)(j != 0 || kk != 0 || l != 0));
          mma_commit2(empty + s);
        }
        mma_commit2(fresh_full);
        if (!ok) break;
      }
      mma_commit2(mma_done);  // no MMA in flight when tensor memory is released (both CTAs)
    } else if (!leader && lane == 0) {
      // forward each stage completed by this CTA's converters to rank 0
      const uint32_t full_b0 = map_to_rank(full_b, 0u);
      for (int i = 0; i < steps; ++i) {
        const int s = i % S;
        if (!mbar_wait(full_b + s, (uint32_t)(i / S) & 1u, P.budget, P.err, abort_s)) break;
        mbar_arrive_cluster(full_b0 + (uint32_t)(s * 8));
      }
    } else if (!leader && lane == 1) {
      // forward each drain completed by this CTA's drainers to rank 0
      const uint32_t fresh_empty0 = map_to_rank(fresh_empty, 0u);
      for (int d = 0; d < drains; ++d) {
        if (!mbar_wait(fresh_empty, (uint32_t)d & 1u, P.budget, P.err, abort_s)) break;
        mbar_arrive_cluster(fresh_empty0);
      }
    }
    __syncwarp();
  } else if (warp >= CONV_WARP0 && warp < CONV_WARP0 + NUM_CONV_WARPS) {
    for (int i = 0; i < steps; ++i) {
      const int s = i % S;
      const uint32_t ph = (uint32_t)(i / S) & 1u;
      if (!warp_wait(full_a + s, ph, P.budget, P.err, abort_s)) break;
      uint8_t *st = smem + s * stage_bytes;
      const int64_t r0 = x_begin + (int64_t)i * BK;
      convert_inplace<TL, L>(reinterpret_cast<const float *>(st + G_HALF_BYTES), st + G_HALF_BYTES, P, col0, r0,
                             warp - CONV_WARP0, lane);
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(full_b + s);
    }
  } else if (warp >= DRAIN_WARP0) {
    const int dw = warp - DRAIN_WARP0;
    const int h = dw >> 2, qd = warp & 3;
    const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
    const uint32_t fresh = tmem + lane_base + (uint32_t)(h * 128);
    const uint32_t run = tmem + lane_base + (uint32_t)(RUN_COL + h * 128);
    const int cc = col0 + qd * 32 + lane;
    const bool own_col = qd * 32 + lane < P.Nt && cc < P.c;
    const float unscale = (own_col && P.colscale != nullptr) ? 1.f / P.colscale[cc] : 1.f;  // a power of two
    const int row0 = mt * BM + h * 128;
    for (int d = 0; d < drains; ++d) {
      if (!warp_wait(fresh_full, (uint32_t)d & 1u, P.budget, P.err, abort_s)) break;
      fence_after();
      drain_once(fresh, run, d == 0, d == drains - 1, own_col, unscale, row0, cc, ch, P, fresh_empty);
    }
  }
  // every MMA of the pair has completed (rank 0's last commit reaches both
  // CTAs) before either CTA releases tensor memory
  if (warp == 1 && lane == 0) drain_wait(mma_done, 0u);
  fence_before();
  __syncthreads();
  cluster_sync();  // no remote arrival or MMA access after this point
  if (warp == 1) {
    fence_after();
    tmem_dealloc2(tmem, 512);
  }
}

template <class TL, int L>
static rhqr_status launch_sketch_pair(dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap &mapX,
                                      const Params &P) {
  RHQR_CUDA_TRY(
      cudaFuncSetAttribute(sketch_tc_pair_kernel<TL, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;  // the pair: the two column tiles (x) of one G tile and K-chunk
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2, grid.x, grid.z);
  cfg.blockDim = dim3(NUM_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  RHQR_CUDA_TRY(cudaLaunchKernelEx(&cfg, sketch_tc_pair_kernel<TL, L>, mapX, P));
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

template <class TL, int L>
static rhqr_status launch_sketch(dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap &mapX, const Params &P) {
  RHQR_CUDA_TRY(cudaFuncSetAttribute(sketch_tc_kernel<TL, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  sketch_tc_kernel<TL, L><<<grid, NUM_THREADS, smem, st>>>(mapX, P);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

// Z[ztop + r, col] = scale * sum_chunk part[chunk][r][col]  (float64, fixed order).
// If a wait of the sketch kernel ran out (*err != 0) its partials are
// incomplete: the sketch rows are set to NaN and RHQR_ETIMEOUT is recorded in
// info (when given), so the failure cannot pass for a result.
__global__ void reduce_part_kernel(const float *part, int32_t nch, int32_t k, int32_t c, int32_t ztop, double scale,
                                   double *Z, int64_t ldz, const int *err, rhqr_info *info) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)k * c) return;
  const bool failed = *err != 0;
  if (failed && idx == 0) set_status(info, RHQR_ETIMEOUT, -1);
  double acc = 0.0;
  for (int ch = 0; ch < nch; ++ch) acc += (double)part[(int64_t)ch * k * c + idx];
  int64_t r = idx / c, col = idx - r * c;
  Z[col * ldz + ztop + r] = failed ? __longlong_as_double(0x7ff8000000000000LL) : acc * scale;
}

// fp16 limbs: f16 keeps 5 exponent bits, so the lower limbs of data of small
// magnitude would fall below its normal range (2^-14) and lose digits.  Each
// column is scaled by the power of two that brings its largest magnitude into
// [2^14, 2^15) before the split (exact), and the partial sums are scaled back.
// The column maxima take one read of X spread over the whole GPU.
// column max |x| over row chunks (grid: columns x chunks), as float bits
// (non-negative floats order like their bit patterns)
__global__ void colmax_kernel(const float *X, int64_t ldx, int64_t n, unsigned int *mx) {
  __shared__ unsigned int bmax;
  if (threadIdx.x == 0) bmax = 0u;
  __syncthreads();
  const float *x = X + (int64_t)blockIdx.x * ldx;
  const int64_t chunk = (n + gridDim.y - 1) / gridDim.y;
  const int64_t r0 = (int64_t)blockIdx.y * chunk, r1 = min(n, r0 + chunk);
  unsigned int local = 0u;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) local = max(local, __float_as_uint(fabsf(x[i])));
  atomicMax(&bmax, local);
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(mx + blockIdx.x, bmax);
}

__global__ void colscale_kernel(const unsigned int *mx, int32_t c, float *scale) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= c) return;
  const float v = __uint_as_float(mx[j]);
  float sc = 1.f;
  if (v > 0.f && isfinite(v)) {
    int e = 0;
    frexpf(v, &e);  // v in [2^(e-1), 2^e)
    sc = ldexpf(1.f, max(-120, min(120, 15 - e)));
  }
  scale[j] = sc;
}

__global__ void copy_top_f32_kernel(const float *X, int64_t ldx, int32_t m, int32_t c, double *Z, int64_t ldz) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * c) return;
  int64_t col = idx / m, i = idx - col * m;
  Z[col * ldz + i] = (double)X[col * ldx + i];
}

// One 16-byte chunk (8 values of one row) per thread: row r, chunk q of the
// operator go to tile (r / 256, q / 8), tile row r % 256, position
// (q % 8) ^ (r % 8); chunks past k or n are written as zeros.
__global__ void operator_tiles_kernel(const uint16_t *G, int64_t ldg, int64_t n, int32_t k, int64_t nkb,
                                      uint4 *Gt) {
  const int64_t nq = nkb * 8;  // chunks per padded row
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t rows = (int64_t)((k + BM - 1) / BM) * BM;
  if (idx >= rows * nq) return;
  const int64_t r = idx / nq, q = idx - r * nq;
  uint4 w;
  if (r < k && q * 8 + 8 <= n) {
    w = *reinterpret_cast<const uint4 *>(G + r * ldg + q * 8);  // rows are 16-byte aligned (ldg)
  } else {
    uint16_t v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int64_t col = q * 8 + e;
      v[e] = (r < k && col < n) ? G[r * ldg + col] : (uint16_t)0;
    }
    w = make_uint4((uint32_t)v[0] | ((uint32_t)v[1] << 16), (uint32_t)v[2] | ((uint32_t)v[3] << 16),
                   (uint32_t)v[4] | ((uint32_t)v[5] << 16), (uint32_t)v[6] | ((uint32_t)v[7] << 16));
  }
  const int64_t tile = (r / BM) * nkb + q / 8;
  const int64_t rr = r % BM;
  Gt[tile * (A_BYTES / 16) + rr * 8 + ((q % 8) ^ (rr % 8))] = w;
}

}  // namespace tc

int64_t operator_tiles_nkb(int64_t n) { return ceil_div(n, (int64_t)tc::BK); }

size_t operator_tiles_bytes(int64_t n, int32_t k) {
  return (size_t)ceil_div((int64_t)k, (int64_t)tc::BM) * (size_t)operator_tiles_nkb(n) * tc::A_BYTES;
}

rhqr_status make_operator_tiles(const void *G, int64_t ldg, int64_t n, int32_t k, void *Gt, cudaStream_t st) {
  if (n < 1 || k < 1 || ldg < n || (ldg * 2) % 16 != 0 || ((uintptr_t)G % 16) != 0) return RHQR_EINVAL;
  const int64_t nkb = operator_tiles_nkb(n);
  const int64_t total = ceil_div((int64_t)k, (int64_t)tc::BM) * tc::BM * nkb * 8;
  tc::operator_tiles_kernel<<<(unsigned)ceil_div(total, (int64_t)256), 256, 0, st>>>((const uint16_t *)G, ldg, n, k,
                                                                                      nkb, (uint4 *)Gt);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

// Work split: the CTAs of one launch cover (k/256) x (c/Nt) tiles times nch
// K-chunks; nch is chosen so the grid fills the 152 SMs in whole waves.
static int64_t tc_nchunks(const SketchView &s, int64_t n, int32_t m, int32_t c, int64_t *kchunk) {
  int64_t K = n - (m & ~63);
  int64_t Np = ceil_div(c, 16) * 16;
  int64_t tiles = ceil_div(s.k, tc::BM) * ceil_div(Np, tc::NT);
  int64_t want = std::max<int64_t>(1, 152 / std::max<int64_t>(1, tiles));
  if (tiles * want < 152) want = ceil_div(152 * ceil_div(tiles, 152), tiles);
  int64_t kc = ceil_div(ceil_div(K, want), tc::KDRAIN) * tc::KDRAIN;
  kc = std::max<int64_t>(kc, tc::KDRAIN);
  if (kchunk) *kchunk = kc;
  return ceil_div(K, kc);
}

bool sketch_tc_supported(const SketchView &s, int64_t n, int32_t m, int32_t c) {
  if (s.kind != RHQR_SKETCH_GAUSSIAN) return false;
  if (s.omega_dtype != RHQR_BF16 && s.omega_dtype != RHQR_F16) return false;
  if (c < 1 || c > tc::MAXC || m < 0 || n <= m || n > (int64_t(1) << 31) - 1) return false;
  if (s.Gt == nullptr || s.gt_nkb != operator_tiles_nkb(n)) return false;
  return tensor_map_encode_fn() != nullptr;
}

size_t sketch_tc_workspace_bytes(const SketchView &s, int64_t n, int32_t m, int32_t c) {
  if (c < 1 || n <= m) return 0;
  return align_up((size_t)tc_nchunks(s, n, m, c, nullptr) * s.k * c * sizeof(float), 256) + 256 +
         align_up((size_t)c * sizeof(float), 256);
}

rhqr_status sketch_apply_tc(const SketchView &s, int32_t m, const float *X, int64_t n, int32_t c, int64_t ldx,
                            int limbs, double *Z, int64_t ldz, void *ws, size_t ws_bytes, rhqr_info *info,
                            long long budget, cudaStream_t st) {
  if (!sketch_tc_supported(s, n, m, c)) return RHQR_ENOTSUP;
  if (limbs < 1 || limbs > 3) return RHQR_EINVAL;
  if ((ldx % 4) != 0 || ((uintptr_t)X % 16) != 0) return RHQR_ENOTSUP;
  int64_t kchunk = 0;
  const int64_t nch = tc_nchunks(s, n, m, c, &kchunk);
  size_t part_bytes = align_up((size_t)nch * s.k * c * sizeof(float), 256);
  const size_t scale_bytes = align_up((size_t)c * sizeof(float), 256);
  if (ws_bytes < part_bytes + 256 + scale_bytes) return RHQR_ENOMEM;
  float *part = (float *)ws;
  int *err = (int *)((char *)ws + part_bytes);
  float *colscale = (float *)((char *)ws + part_bytes + 256);
  RHQR_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  const bool scaled = s.omega_dtype == RHQR_F16;
  if (scaled) {
    unsigned int *mx = reinterpret_cast<unsigned int *>(colscale);  // maxima first, then the scales in place
    RHQR_CUDA_TRY(cudaMemsetAsync(mx, 0, (size_t)c * sizeof(unsigned int), st));
    const unsigned chunks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(152 * 8, c), ceil_div(n, 4096)));
    tc::colmax_kernel<<<dim3((unsigned)c, chunks), 256, 0, st>>>(X, ldx, n, mx);
    RHQR_LAUNCH_CHECK();
    tc::colscale_kernel<<<(unsigned)ceil_div(c, 256), 256, 0, st>>>(mx, c, colscale);
    RHQR_LAUNCH_CHECK();
  }

  const int32_t Np = (int32_t)ceil_div(c, 16) * 16;
  const int32_t Nt = std::min<int32_t>(tc::NT, Np);
  CUtensorMap mapX;
  {
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)c};
    cuuint64_t strides[1] = {(cuuint64_t)ldx * 4};
    cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)Nt};
    cuuint32_t estr[2] = {1, 1};
    CUresult cr = tensor_map_encode_fn()(&mapX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(X), dims,
                                       strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return RHQR_ECUDA;
  }

  tc::Params P;
  P.n = n;
  P.m = m;
  P.m64 = m & ~63;
  P.c = c;
  P.Nt = Nt;
  P.k = s.k;
  P.kchunk = kchunk;
  P.limbs = limbs;
  P.stages = limbs <= 2 ? 3 : 2;
  P.kdrain = tc::KDRAIN;
  P.xbytes = tc::BK * Nt * 4;
  P.part = part;
  P.gt = (const char *)s.Gt;
  P.gt_nkb = s.gt_nkb;
  P.colscale = scaled ? colscale : nullptr;
  P.err = err;
  P.budget = budget > 0 ? budget : kDefaultWaitBudget;
  const size_t stage_bytes = tc::A_BYTES + tc::X_BYTES + (limbs <= 2 ? 0 : (size_t)limbs * tc::B_BYTES);
  size_t smem = 1024 + (size_t)P.stages * stage_bytes + 256;
  dim3 grid((unsigned)ceil_div(s.k, tc::BM), (unsigned)ceil_div(Np, Nt), (unsigned)nch);
  if (grid.y == 2 && limbs <= 2) {
    // two column tiles: CTA pairs sharing each G tile (cta_group::2)
    P.stages = tc::PAIR_STAGES;
    const size_t smem2 = 1024 + (size_t)tc::PAIR_STAGES * (tc::G_HALF_BYTES + tc::X_BYTES) + 256;
    if (s.omega_dtype == RHQR_BF16) {
      if (limbs == 1) RHQR_TRY((tc::launch_sketch_pair<__nv_bfloat16, 1>(grid, smem2, st, mapX, P)));
      else RHQR_TRY((tc::launch_sketch_pair<__nv_bfloat16, 2>(grid, smem2, st, mapX, P)));
    } else {
      if (limbs == 1) RHQR_TRY((tc::launch_sketch_pair<__half, 1>(grid, smem2, st, mapX, P)));
      else RHQR_TRY((tc::launch_sketch_pair<__half, 2>(grid, smem2, st, mapX, P)));
    }
  } else if (s.omega_dtype == RHQR_BF16) {
    switch (limbs) {
      case 1: RHQR_TRY((tc::launch_sketch<__nv_bfloat16, 1>(grid, smem, st, mapX, P))); break;
      case 2: RHQR_TRY((tc::launch_sketch<__nv_bfloat16, 2>(grid, smem, st, mapX, P))); break;
      default: RHQR_TRY((tc::launch_sketch<__nv_bfloat16, 3>(grid, smem, st, mapX, P))); break;
    }
  } else {
    switch (limbs) {
      case 1: RHQR_TRY((tc::launch_sketch<__half, 1>(grid, smem, st, mapX, P))); break;
      case 2: RHQR_TRY((tc::launch_sketch<__half, 2>(grid, smem, st, mapX, P))); break;
      default: RHQR_TRY((tc::launch_sketch<__half, 3>(grid, smem, st, mapX, P))); break;
    }
  }
  if (m > 0) {
    tc::copy_top_f32_kernel<<<(unsigned)ceil_div((int64_t)m * c, 256), 256, 0, st>>>(X, ldx, m, c, Z, ldz);
    RHQR_LAUNCH_CHECK();
  }
  int64_t tot = (int64_t)s.k * c;
  tc::reduce_part_kernel<<<(unsigned)ceil_div(tot, 256), 256, 0, st>>>(part, (int32_t)nch, s.k, c, m,
                                                                       1.0 / sqrt((double)s.k), Z, ldz, err, info);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

}  // namespace rhqr
