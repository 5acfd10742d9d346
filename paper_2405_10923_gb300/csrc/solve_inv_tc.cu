// Q = X Tri^{-1} for float32 X (n x m, m <= 256) on the tcgen05 tensor cores,
// through the explicit inverse computed on the small side in float64:
//   Tri^{-1} = D (I + F),  D = diag(Tri^{-1}),  F = D^{-1} E strictly upper,
//   Y = A (I + F)  with  A = X D.
// With Tri = R this forms recRHQR's Q = W R^{-1} (Section 3.3).  The loaders
// scale X by D in float32 and split A into three bf16 limbs (float32 values
// are sums of three bf16 numbers); (I + F) is split into three bf16 limbs with
// its unit diagonal exact.  For a column chunk, the products of the row chunk
// that holds its diagonal come last and within them the big limb product
// last, so the float32 accumulator only holds A F -- small next to Y in
// refinement passes, where Tri is close to a signed identity -- until A itself
// arrives.  Six limb products (weight >= 2^-16) are taken when F is not small,
// three (plus A's smallest limb through the diagonal) when F is small enough
// that the dropped ones stay below float32 rounding; either way into one
// float32 accumulator per buffer, so the accumulators are double-buffered and
// the epilogue of a tile overlaps the MMAs of the next.
//
// Tiles of 128 rows.  Columns are grouped in chunks of 64; row chunk kc of
// (I + F) feeds the column chunks c >= kc, one MMA group per row chunk.  For
// m > 128 the column chunks are shared between the two CTAs of a cluster,
// balanced by tensor work ({0, 3} and {1, 2} for four chunks; {2} and {0, 1}
// for three); each CTA keeps its blocks of (I + F) in shared memory as B
// operands.  Tensor memory per CTA: two A stages (one 64-column chunk, three
// limbs x 32 columns) and two accumulators of up to 128 columns (a double
// buffer).  For an in-place solve a CTA
// stores its columns of a tile only after the peer CTA's loaders have read the
// tile (counters in its shared memory that the peer increments).
//
// Warp roles: warp 0 issues the MMAs (one thread), warp 1 owns tensor memory,
// warp 2 loads X by TMA (64-column boxes of a tile, two stages, each box of the
// next tile prefetched into L2 when this one is loaded) when X and its
// leading dimension are 16-byte aligned, warps 4-11 (two groups, one per A
// stage) scale, split and store the limbs to tensor memory (thread = row =
// tensor-memory lane), warps 12-15 drain the accumulator into shared memory
// in pieces of 32 columns that one thread writes to Y with TMA stores (or,
// when Y is not 16-byte aligned, store Y column by column).  Every wait is
// bounded.
#include <algorithm>
#include <cstring>

#include "solve_inv_tc.cuh"
#include "tcgen05.cuh"
#include "tma_host.cuh"

namespace rhqr {

// ---- small side: R^{-1} ----------------------------------------------------
// Column j of Rinv solves R x = e_j by a backward column sweep (one warp per
// column): once x_l is known, the partial sums s_i (i < l) take R_il x_l and
// x_{l-1} = -s_{l-1} / R_{l-1,l-1}.
__global__ void upper_inverse_kernel(const double *R, int32_t m, double *Rinv) {
  // one warp per column, the longest sweeps (largest j) first
  const int jj = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (jj >= m) return;
  const int j = m - 1 - jj;
  column_sweep<4>(R, m, m, j, 1.0 / R[(int64_t)j * m + j], nullptr, true, Rinv + (int64_t)j * m);
}

rhqr_status upper_inverse(const double *R, int32_t m, double *Rinv, cudaStream_t st) {
  if (m < 1 || m > 256) return RHQR_ENOTSUP;
  upper_inverse_kernel<<<(unsigned)m, 32, 0, st>>>(R, m, Rinv);  // spread over the SMs (FP64 issue-bound)
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

namespace sit {

constexpr int TILE = 128;
constexpr int NUM_THREADS = 512;
constexpr int LOAD_WARP0 = 4;  // two groups of four loader warps, one per A stage
constexpr int EPI_WARP0 = 12;
constexpr int A_COLS = 96;     // one A stage: 3 limbs x 32 columns (64 bf16 per lane)
constexpr int ACC_COL0 = 2 * A_COLS;
constexpr int MAX_W = 128;     // accumulator columns of one CTA (2 buffers + 2 A stages <= 512)
constexpr int MAXM = 256;
constexpr int MAXG = 8;        // MMA groups per CTA
constexpr int XST_BYTES = TILE * 64 * 4;  // one TMA stage of X: 128 rows x 64 columns float32
constexpr int YST_BYTES = TILE * 32 * 4;  // one piece of Q for a TMA store: 128 rows x 32 columns
constexpr size_t SMEM_LIMIT = 227 * 1024;
static_assert(NUM_THREADS == 512, "roles: warps 0-3 control, 4-11 loaders, 12-15 epilogue");

// One MMA group: row chunk kc of F times the columns [c0, c0 + N) of this CTA.
// Row chunk kc of (I + F) times the CTA's columns of chunks >= kc: they occupy
// the accumulator columns [acc, acc + N) (owned chunks in order).
struct Grp {
  int32_t kc, N, acc;  // acc: first accumulator column
  int32_t boff;        // byte offset of the three limb blocks (N rows x 128 bytes each)
  int32_t diag;        // chunk kc is owned: the block holds the identity's diagonal
};

struct CtaPlan {
  int32_t ngrp, nk;         // groups; row chunks to load (0 .. nk-1)
  Grp g[MAXG];
  int32_t ncc, cc[2], cc_acc[2], cc_w[2];  // owned column chunks: index, accumulator column, width
  int32_t bbytes;
};

struct Params {
  const float *X;
  int64_t ldx;
  float *Y;
  int64_t ldy;
  int64_t nrows;
  int32_t m, nprod, split, bregion;  // nprod: 6, 3, or 0 = chosen from max |F|
  int32_t use_tma;                   // X staged by TMA (16-byte aligned X and ld), else column loads
  int32_t use_tma_y;                 // Q written by TMA stores from shared memory, else column stores
  const double *Rinv;
  CtaPlan plan[2];
  rhqr_info *info;
  long long budget;
};

// three bf16 limbs of two float32 values at once (packed conversions; a low, b high)
__device__ __forceinline__ void split3_pair(float a, float b, uint32_t &w0, uint32_t &w1, uint32_t &w2) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const float ra = a - hf.x, rb = b - hf.y;
  const __nv_bfloat162 mi = __floats2bfloat162_rn(ra, rb);
  const float2 mf = __bfloat1622float2(mi);
  const __nv_bfloat162 lo = __floats2bfloat162_rn(ra - mf.x, rb - mf.y);
  w0 = *reinterpret_cast<const uint32_t *>(&h);
  w1 = *reinterpret_cast<const uint32_t *>(&mi);
  w2 = *reinterpret_cast<const uint32_t *>(&lo);
}
__device__ __forceinline__ void split3d(double x, __nv_bfloat16 &h, __nv_bfloat16 &mi, __nv_bfloat16 &lo) {
  h = __double2bfloat16(x);
  const double r1 = x - (double)__bfloat162float(h);
  mi = __double2bfloat16(r1);
  lo = __double2bfloat16(r1 - (double)__bfloat162float(mi));
}

// Limb products of A F: the dropped ones (weight 2^-16) stay below float32
// rounding of Y when 3 sqrt(m) max |F| <= 2^-8.
__device__ __forceinline__ int choose_nprod(int forced, int m, float fmax) {
  if (forced != 0) return forced;
  return 3.f * sqrtf((float)m) * fmax <= 0.00390625f ? 3 : 6;
}

// The MMAs of one group, smallest limb products first, fully unrolled:
//   NPROD 3: (1,0) (0,1) (0,0)          [A limb, (I + F) limb]
//   NPROD 4: (2,0) (1,0) (0,1) (0,0)    (the group holds a diagonal block: all
//                                        three limbs of A pass through the identity)
//   NPROD 6: (2,0) (1,1) (0,2) (1,0) (0,1) (0,0)
template <int NPROD>
__device__ __forceinline__ void issue_group(uint32_t dcol, uint32_t a_stage, uint32_t dhi, uint32_t blo,
                                            uint32_t lstride, uint32_t idesc, bool first) {
  constexpr int PA3[3] = {1, 0, 0}, PB3[3] = {0, 1, 0};
  constexpr int PA4[4] = {2, 1, 0, 0}, PB4[4] = {0, 0, 1, 0};
  constexpr int PA6[6] = {2, 1, 0, 1, 0, 0}, PB6[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
  for (int pr = 0; pr < NPROD; ++pr) {
    const int pa = NPROD == 3 ? PA3[pr] : NPROD == 4 ? PA4[pr] : PA6[pr];
    const int pb = NPROD == 3 ? PB3[pr] : NPROD == 4 ? PB4[pr] : PB6[pr];
    const uint32_t lo = blo + (uint32_t)pb * lstride;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      // the first MMA into an accumulator of row chunk 0 starts the sums
      const uint32_t accumulate = (!first || kk > 0 || pr > 0) ? 1u : 0u;
      tc::mma_ts(dcol, a_stage + (uint32_t)(pa * 32 + kk * 8), ((uint64_t)dhi << 32) | (lo + 2u * kk), idesc,
                 accumulate);
    }
  }
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    solve_inv_tc_kernel(const __grid_constant__ Params P, const __grid_constant__ CUtensorMap tmapX,
                        const __grid_constant__ CUtensorMap tmapY32, const __grid_constant__ CUtensorMap tmapY16) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *bsm = smem;                                         // (I + F) blocks
  float *xst = reinterpret_cast<float *>(smem + P.bregion);    // 2 TMA stages [col][row]
  float *ybuf = xst + 2 * (XST_BYTES / 4);                     // 2 pieces of Q [col][row]
  float *dvec = ybuf + 2 * (YST_BYTES / 4);
  uint64_t *bars = reinterpret_cast<uint64_t *>(dvec + MAXM);
  // accumulator barriers per buffer b and owned column chunk ci: [2 b + ci]
  uint64_t *a_full = bars, *a_empty = bars + 2, *acc_full = bars + 4, *acc_empty = bars + 8;
  uint64_t *x_full = bars + 12, *x_empty = bars + 14;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 17);
  volatile int *abort_s = reinterpret_cast<volatile int *>(tmem_slot + 1);
  int *err_s = reinterpret_cast<int *>(tmem_slot + 2);
  unsigned int *fmax_s = tmem_slot + 3;  // max |F| of this CTA's blocks (float bits, >= 0)
  uint32_t *peer_cnt = tmem_slot + 4;    // [2]: rows read by the peer's loader groups
  uint64_t *mma_done = bars + 16;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = P.split ? tc::cluster_ctarank() : 0u;
  const CtaPlan &C = P.plan[rank];
  const int m = P.m;

  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(a_full + s, 4);
      tc::mbar_init(a_empty + s, 1);
      for (int ci = 0; ci < 2; ++ci) {
        tc::mbar_init(acc_full + 2 * s + ci, 1);
        tc::mbar_init(acc_empty + 2 * s + ci, 4);
      }
      tc::mbar_init(x_full + s, 1);
      tc::mbar_init(x_empty + s, 4);
    }
    tc::mbar_init(mma_done, 1);
    *abort_s = 0;
    *err_s = 0;
    *fmax_s = 0u;
    peer_cnt[0] = 0;
    peer_cnt[1] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // ---- B operands: (I + F) blocks (group g, limb l: N rows = the group's
  //      columns j, 64 K values = rows 64 kc .. 64 kc + 63), and D.  Entry
  //      (i, j): F_ij = Rinv_ij / Rinv_ii for i < j, 1 for i = j (exact in bf16).
  float fmax = 0.f;
  for (int gi = 0; gi < C.ngrp; ++gi) {
    const Grp &G = C.g[gi];
    uint8_t *blk = bsm + G.boff;
    for (int q = threadIdx.x; q < G.N * 8; q += NUM_THREADS) {
      const int nrow = q >> 3, chunk = q & 7;
      const int a = G.acc + nrow;  // accumulator column -> global column j
      int ci = 0;
      while (ci + 1 < C.ncc && a >= C.cc_acc[ci + 1]) ++ci;
      const int j = 64 * C.cc[ci] + (a - C.cc_acc[ci]);
      uint32_t w[3][4];
#pragma unroll
      for (int e2 = 0; e2 < 4; ++e2) {
        double f[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int i = 64 * G.kc + chunk * 8 + 2 * e2 + h;
          f[h] = 0.0;
          if (j < m && i < j) {
            f[h] = P.Rinv[(int64_t)j * m + i] / P.Rinv[(int64_t)i * m + i];
            fmax = fmaxf(fmax, (float)fabs(f[h]));
          } else if (j < m && i == j) {
            f[h] = 1.0;
          }
        }
        __nv_bfloat16 ah, am, al, bh, bm, bl;
        split3d(f[0], ah, am, al);
        split3d(f[1], bh, bm, bl);
        w[0][e2] = tc::pack_bf16(ah, bh);
        w[1][e2] = tc::pack_bf16(am, bm);
        w[2][e2] = tc::pack_bf16(al, bl);
      }
      const uint32_t off = tc::sw128_offset((uint32_t)nrow, (uint32_t)chunk);
#pragma unroll
      for (int l = 0; l < 3; ++l)
        *reinterpret_cast<uint4 *>(blk + (size_t)l * G.N * 128 + off) = make_uint4(w[l][0], w[l][1], w[l][2], w[l][3]);
    }
  }
  for (int j = threadIdx.x; j < MAXM; j += NUM_THREADS) dvec[j] = j < m ? (float)P.Rinv[(int64_t)j * m + j] : 0.f;
  fmax = fmaxf(fmax, __shfl_xor_sync(0xffffffffu, fmax, 16));
  fmax = fmaxf(fmax, __shfl_xor_sync(0xffffffffu, fmax, 8));
  fmax = fmaxf(fmax, __shfl_xor_sync(0xffffffffu, fmax, 4));
  fmax = fmaxf(fmax, __shfl_xor_sync(0xffffffffu, fmax, 2));
  fmax = fmaxf(fmax, __shfl_xor_sync(0xffffffffu, fmax, 1));
  if (lane == 0) atomicMax(fmax_s, __float_as_uint(fmax));
  tc::fence_proxy_async();
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, 512);
    tc::tmem_relinquish();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (P.split) tc::cluster_sync();  // the peer's counters are initialised before anyone adds to them
  const uint32_t tmem = *tmem_slot;

  const int64_t ntiles = (P.nrows + TILE - 1) / TILE;
  const int64_t t0 = P.split ? (int64_t)(blockIdx.x >> 1) : (int64_t)blockIdx.x;
  const int64_t tstep = P.split ? (int64_t)(gridDim.x >> 1) : (int64_t)gridDim.x;

  // Six products when F is not small (e.g. the first pass of an
  // ill-conditioned W), three otherwise; one accumulator, double-buffered.
  const int nprod = choose_nprod(P.nprod, m, __uint_as_float(*fmax_s));
  constexpr uint32_t nbuf = 2;

  if (warp == 0) {
    if (lane == 0) {
      const uint32_t dhi = (uint32_t)(tc::sw128_desc(tc::smem_u32(bsm)) >> 32);
      const uint32_t bsm_lo = (uint32_t)tc::sw128_desc(tc::smem_u32(bsm));
      uint32_t gch = 0;
      bool ok = true;
      uint32_t it = 0;
      for (int64_t t = t0; t < ntiles && ok; t += tstep, ++it) {
        const uint32_t b = it % nbuf, u = it / nbuf;
        // the first group writes every owned chunk: all of them drained
        for (int ci = 0; ci < C.ncc && ok; ++ci)
          ok = tc::mbar_wait(acc_empty + 2 * b + ci, (u & 1u) ^ 1u, P.budget, err_s, abort_s);
        if (!ok) break;
        tc::fence_after();
        const uint32_t acc = tmem + (uint32_t)(ACC_COL0 + b * MAX_W);
        for (int kc = 0; kc < C.nk; ++kc, ++gch) {
          const uint32_t s = gch & 1u;
          if (!tc::mbar_wait(a_full + s, (gch >> 1) & 1u, P.budget, err_s, abort_s)) {
            ok = false;
            break;
          }
          tc::fence_after();
          const Grp &G = C.g[kc];  // one group per row chunk
          const uint32_t a_stage = tmem + (uint32_t)(s * A_COLS);
          const uint32_t dcol = acc + (uint32_t)G.acc;
          const uint32_t blo = bsm_lo + (uint32_t)(G.boff >> 4), lstride = (uint32_t)G.N * 8u;
          const uint32_t idesc = tc::idesc_bf16(128, G.N);
          const bool first = G.kc == 0;
          if (nprod == 6) issue_group<6>(dcol, a_stage, dhi, blo, lstride, idesc, first);
          else if (G.diag) issue_group<4>(dcol, a_stage, dhi, blo, lstride, idesc, first);
          else issue_group<3>(dcol, a_stage, dhi, blo, lstride, idesc, first);
          tc::mma_commit(a_empty + s);
        }
        if (!ok) break;
        // the tile is handed over whole (the next tile's MMAs use the other buffer)
        tc::mma_commit(acc_full + 2 * b);
      }
      tc::mma_quiesce(mma_done);  // no MMA in flight when tensor memory is released
    }
    __syncwarp();
  } else if (warp == 2) {
    if (lane == 0 && P.use_tma) {
      // TMA producer: chunk G of the tile sequence goes to stage G & 1 (loader group G & 1)
      uint32_t G = 0;
      int last_u[2] = {-1, -1};  // use index of the last copy issued into each stage
      bool ok = true;
      for (int64_t t = t0; t < ntiles && ok; t += tstep)
        for (int kc = 0; kc < C.nk; ++kc, ++G) {
          const uint32_t s = G & 1u, u = G >> 1;
          if (!tc::mbar_wait(x_empty + s, (u & 1u) ^ 1u, P.budget, err_s, abort_s)) {
            ok = false;
            break;
          }
          tc::mbar_expect_tx(x_full + s, (uint32_t)XST_BYTES);
          tc::tma_load_2d(xst + s * (XST_BYTES / 4), &tmapX, x_full + s, (int)(t * TILE), kc * 64);
          last_u[s] = (int)u;
          // two shared-memory stages hold too few bytes to cover DRAM latency: the
          // same chunk of this CTA's next tile is brought into L2 a tile ahead
          if (t + tstep < ntiles) tc::tma_prefetch_2d(&tmapX, (int)((t + tstep) * TILE), kc * 64);
        }
      // the last copy into each stage completes before the CTA exits (already so
      // on the normal path; after a stop it may still be in flight)
      for (int s = 0; s < 2; ++s)
        if (last_u[s] >= 0) tc::drain_wait(x_full + s, (uint32_t)last_u[s] & 1u);
    }
    __syncwarp();
  } else if (warp >= LOAD_WARP0 && warp < EPI_WARP0) {
    // Loader group grp handles the chunks of even / odd global index, i.e. A
    // stage grp; group 0 also prefetches the next tile of X into L2.
    const int grp = (warp - LOAD_WARP0) >> 2;
    const int qd = warp & 3;
    const int r = qd * 32 + lane;
    const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
    const uint32_t peer_addr = P.split ? tc::map_to_rank(peer_cnt + grp, rank ^ 1u) : 0u;
    const int ncols = C.nk * 64 < m ? C.nk * 64 : m;
    uint32_t gch = 0;
    bool ok = true;
    for (int64_t t = t0; t < ntiles && ok; t += tstep) {
      const int64_t row = t * TILE + r;
      const bool live = row < P.nrows;
      if (!P.use_tma && grp == 0 && t + tstep < ntiles) {
        // one 128-byte line per column and warp: lane l takes columns l, l + 32, ...
        const int64_t r0 = (t + tstep) * TILE + qd * 32;
        const int64_t rl = r0 + 31 < P.nrows ? r0 + 31 : P.nrows - 1;
        if (r0 < P.nrows)
          for (int col = lane; col < ncols; col += 32) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(P.X + (int64_t)col * P.ldx + r0));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(P.X + (int64_t)col * P.ldx + rl));
          }
      }
      for (int kc = 0; kc < C.nk; ++kc, ++gch) {
        if ((int)(gch & 1u) != grp) continue;
        float v[64];
        const uint32_t s = (uint32_t)grp, u = gch >> 1;
        if (P.use_tma) {
          if (!tc::warp_wait(x_full + s, u & 1u, P.budget, err_s, abort_s)) {
            ok = false;
            break;
          }
          const float *xs = xst + s * (XST_BYTES / 4);
#pragma unroll
          for (int c = 0; c < 64; ++c) v[c] = xs[c * TILE + r];  // zero beyond the rows / columns of X
          // the stage is refilled by TMA (async proxy) after this release: the fence
          // completes these shared-memory reads before any lane signals it
          tc::fence_proxy_async();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(x_empty + s);
        } else {
#pragma unroll
          for (int c = 0; c < 64; ++c) {
            const int col = kc * 64 + c;
            v[c] = (live && col < m) ? __ldg(P.X + (int64_t)col * P.ldx + row) : 0.f;
          }
        }
        if (!tc::warp_wait(a_empty + s, (u & 1u) ^ 1u, P.budget, err_s, abort_s)) {
          ok = false;
          break;
        }
        tc::fence_after();
#pragma unroll
        for (int pc = 0; pc < 4; ++pc) {
          uint32_t w0[8], w1[8], w2[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int c = 16 * pc + 2 * j;
            split3_pair(v[c] * dvec[kc * 64 + c], v[c + 1] * dvec[kc * 64 + c + 1], w0[j], w1[j], w2[j]);
          }
          const uint32_t col = tmem + lane_base + (uint32_t)(s * A_COLS + pc * 8);
          tc::tmem_st8(col, w0);
          tc::tmem_st8(col + 32u, w1);
          tc::tmem_st8(col + 64u, w2);
        }
        tc::tmem_wait_st();
        tc::fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(a_full + s);
      }
      // this lane has read its row of the tile: tell the peer CTA
      if (ok && P.split) tc::remote_add_release(peer_addr, 1u);
    }
  } else if (warp >= EPI_WARP0) {
    const int qd = warp & 3;
    const int r = qd * 32 + lane;
    const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
    uint32_t it = 0, piece = 0;
    bool ok_all = true;
    for (int64_t t = t0; t < ntiles && ok_all; t += tstep, ++it) {
      const uint32_t b = it % nbuf, u = it / nbuf;
      const int64_t row = t * TILE + r;
      const bool live = row < P.nrows;
      const bool issuer = qd == 0 && lane == 0;  // the epilogue thread that issues TMA stores
      // the owned chunks of the tile (one commit for the whole tile); each
      // one's accumulator columns are released as soon as they have been read
      for (int ci = 0; ci < C.ncc; ++ci) {
        bool okw = true;
        if (ci == 0) okw = tc::mbar_wait(acc_full + 2 * b, u & 1u, P.budget, err_s, abort_s);
        okw = __all_sync(0xffffffffu, okw);
        // the four epilogue warps share named barriers: they stop together
        if (P.use_tma_y) okw = tc::named_and(1, 128, okw);
        if (!okw) {
          ok_all = false;
          break;
        }
        tc::fence_after();
        // the peer's loaders must be done with this tile: in place, before it is
        // overwritten; otherwise it keeps the pair within a tile of each other,
        // so both CTAs read each X tile from L2 (without it the first,
        // not-in-place pass read 1.66x the algorithmic bytes from DRAM)
        if (ci == 0 && P.split) {
          const uint32_t need = 128u * (uint32_t)(it + 1);
          long long spins = 0;
          bool ok = true;
          while (tc::ld_acquire_cluster(peer_cnt) < need || tc::ld_acquire_cluster(peer_cnt + 1) < need) {
            if (*abort_s) {
              ok = false;
              break;
            }
            if (++spins > P.budget) {
              atomicExch(err_s, 1);
              *abort_s = 1;
              ok = false;
              break;
            }
          }
          ok = __all_sync(0xffffffffu, ok);
          if (P.use_tma_y) ok = tc::named_and(1, 128, ok);
          if (!ok) {
            ok_all = false;
            break;
          }
        }
        if (P.use_tma_y) {
          // pieces of 32 (or a last 16) columns: TMEM -> shared memory -> one TMA store
          for (int c0 = 0; c0 < C.cc_w[ci]; c0 += 32, ++piece) {
            const int wc = C.cc_w[ci] - c0 >= 32 ? 32 : 16;
            float *yb = ybuf + (piece & 1u) * (YST_BYTES / 4);
            if (issuer) tc::bulk_wait_read_1();  // the store that used this buffer has read it
            tc::named_sync(1, 128);
            for (int h = 0; h < wc / 16; ++h) {
              const uint32_t col =
                  tmem + lane_base + (uint32_t)(ACC_COL0 + b * MAX_W + C.cc_acc[ci] + c0 + 16 * h);
              uint32_t a0[16];
              tc::tmem_ld16(col, a0);
              tc::tmem_wait_ld();
#pragma unroll
              for (int j = 0; j < 16; ++j) yb[(16 * h + j) * TILE + r] = __uint_as_float(a0[j]);
            }
            tc::fence_proxy_async();
            tc::named_sync(1, 128);
            if (issuer) {
              tc::tma_store_2d(wc == 32 ? (const void *)&tmapY32 : (const void *)&tmapY16, yb, (int)(t * TILE),
                               C.cc[ci] * 64 + c0);
              tc::bulk_commit();
            }
          }
        } else {
          for (int cb = 0; cb < C.cc_w[ci] / 16; ++cb) {
            const uint32_t col = tmem + lane_base + (uint32_t)(ACC_COL0 + b * MAX_W + C.cc_acc[ci] + cb * 16);
            uint32_t a0[16];
            tc::tmem_ld16(col, a0);
            tc::tmem_wait_ld();
            if (live) {
              const int col0 = C.cc[ci] * 64 + cb * 16;
              float *y = P.Y + (int64_t)col0 * P.ldy + row;
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const float v = __uint_as_float(a0[j]);
                if (col0 + j < m) y[(int64_t)j * P.ldy] = v;
              }
            }
          }
        }
        tc::fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(acc_empty + 2 * b + ci);
      }
    }
    if (P.use_tma_y && qd == 0 && lane == 0) tc::bulk_wait_all();  // stores complete before exit
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
  if (P.split) tc::cluster_sync();  // no peer adds into this CTA's shared memory after it exits
  if (threadIdx.x == 0 && *err_s) set_status(P.info, RHQR_ETIMEOUT, -1);
}

// Plan of one CTA owning column chunks `own` (sorted) of mp columns.
static bool make_plan(const int *own, int nown, int mp, CtaPlan &C) {
  C = CtaPlan{};
  int acc = 0;
  for (int i = 0; i < nown; ++i) {
    C.cc[i] = own[i];
    C.cc_acc[i] = acc;
    C.cc_w[i] = std::min(64, mp - 64 * own[i]);
    acc += C.cc_w[i];
  }
  C.ncc = nown;
  if (acc > MAX_W) return false;
  C.nk = own[nown - 1] + 1;
  if (C.nk > MAXG) return false;
  int off = 0;
  for (int kc = 0; kc < C.nk; ++kc) {
    // the owned chunks c >= kc are a suffix of the owned list: one group
    int i = 0;
    while (i < nown && own[i] < kc) ++i;
    Grp &G = C.g[C.ngrp++];
    G.kc = kc;
    G.acc = C.cc_acc[i];
    G.N = acc - C.cc_acc[i];
    G.boff = off;
    off += 3 * G.N * 128;
    G.diag = 0;
    for (int q = i; q < nown; ++q)
      if (own[q] == kc) G.diag = 1;
  }
  C.bbytes = off;
  return true;
}

static size_t smem_bytes(int bregion) {
  return 1024 + (size_t)bregion + 2 * XST_BYTES + 2 * YST_BYTES + MAXM * 4 + 21 * 8 + 64;
}

// Column chunks of the one or two CTAs per tile and the shared-memory size.
static bool plan(int32_t m, Params &P, size_t *smem) {
  if (m < 1 || m > MAXM) return false;
  const int mp = (int)ceil_div(m, 16) * 16;
  const int nc = (mp + 63) / 64;
  bool ok;
  if (nc <= 2) {
    const int own[2] = {0, 1};
    P.split = 0;
    ok = make_plan(own, nc, mp, P.plan[0]);
    P.plan[1] = P.plan[0];
  } else if (nc == 3) {
    const int a[1] = {2}, b[2] = {0, 1};
    P.split = 1;
    ok = make_plan(a, 1, mp, P.plan[0]) && make_plan(b, 2, mp, P.plan[1]);
  } else {
    const int a[2] = {0, 3}, b[2] = {1, 2};
    P.split = 1;
    ok = make_plan(a, 2, mp, P.plan[0]) && make_plan(b, 2, mp, P.plan[1]);
  }
  if (!ok) return false;
  P.bregion = (int32_t)align_up((size_t)std::max(P.plan[0].bbytes, P.plan[1].bbytes), 1024);
  *smem = smem_bytes(P.bregion);
  return *smem <= SMEM_LIMIT;
}

}  // namespace sit

bool solve_inv_tc_supported(int32_t m) {
  sit::Params P;
  size_t smem = 0;
  return sit::plan(m, P, &smem);
}

rhqr_status rows_solve_inv_tc(const float *X, int64_t ldx, int64_t nrows, int32_t m, const double *Rinv, int nprod,
                              float *Y, int64_t ldy, rhqr_info *info, long long budget, cudaStream_t st) {
  if (nrows <= 0) return RHQR_OK;
  if (nprod != 6 && nprod != 3 && nprod != 0) return RHQR_EINVAL;
  if ((X == Y && ldx != ldy) || ldx < nrows || ldy < nrows) return RHQR_EINVAL;
  sit::Params P;
  size_t smem = 0;
  if (!sit::plan(m, P, &smem)) return RHQR_ENOTSUP;
  P.X = X;
  P.ldx = ldx;
  P.Y = Y;
  P.ldy = ldy;
  P.nrows = nrows;
  P.m = m;
  P.nprod = nprod;
  P.Rinv = Rinv;
  P.info = info;
  P.budget = budget;
  CUtensorMap mapX;
  std::memset(&mapX, 0, sizeof(mapX));
  P.use_tma = 0;
  if ((ldx % 4) == 0 && ((uintptr_t)X % 16) == 0 && nrows < ((int64_t)1 << 31) - sit::TILE &&
      tensor_map_encode_fn() != nullptr) {
    cuuint64_t dims[2] = {(cuuint64_t)nrows, (cuuint64_t)m};
    cuuint64_t strides[1] = {(cuuint64_t)ldx * 4};
    cuuint32_t box[2] = {(cuuint32_t)sit::TILE, 64u};
    cuuint32_t estr[2] = {1, 1};
    if (tensor_map_encode_fn()(&mapX, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(X), dims, strides, box,
                               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
      P.use_tma = 1;
  }
  CUtensorMap mapY32, mapY16;
  std::memset(&mapY32, 0, sizeof(mapY32));
  std::memset(&mapY16, 0, sizeof(mapY16));
  P.use_tma_y = 0;
  if (P.use_tma && (ldy % 4) == 0 && ((uintptr_t)Y % 16) == 0) {
    cuuint64_t dims[2] = {(cuuint64_t)nrows, (cuuint64_t)m};
    cuuint64_t strides[1] = {(cuuint64_t)ldy * 4};
    cuuint32_t estr[2] = {1, 1};
    cuuint32_t box32[2] = {(cuuint32_t)sit::TILE, 32u}, box16[2] = {(cuuint32_t)sit::TILE, 16u};
    auto enc = tensor_map_encode_fn();
    if (enc(&mapY32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, Y, dims, strides, box32, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS &&
        enc(&mapY16, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, Y, dims, strides, box16, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
            CUDA_SUCCESS)
      P.use_tma_y = 1;
  }
  static bool attr_set = false;
  static int sms = 0;
  if (!attr_set) {
    RHQR_CUDA_TRY(cudaFuncSetAttribute(sit::solve_inv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sit::SMEM_LIMIT));
    int dev = 0;
    RHQR_CUDA_TRY(cudaGetDevice(&dev));
    RHQR_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    attr_set = true;
  }
  const int64_t ntiles = ceil_div(nrows, sit::TILE);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.blockDim = dim3(sit::NUM_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  if (P.split) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    static int max_clusters = 0;
    if (max_clusters == 0) {
      cfg.gridDim = dim3(2 * (unsigned)(sms / 2), 1, 1);
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, sit::solve_inv_tc_kernel, &cfg) != cudaSuccess || n < 1) {
        (void)cudaGetLastError();
        n = sms / 2;
      }
      max_clusters = n;
    }
    cfg.gridDim = dim3(2 * (unsigned)std::min<int64_t>(ntiles, max_clusters), 1, 1);
  } else {
    cfg.attrs = nullptr;
    cfg.numAttrs = 0;
    cfg.gridDim = dim3((unsigned)std::min<int64_t>(ntiles, sms), 1, 1);
  }
  RHQR_CUDA_TRY(cudaLaunchKernelEx(&cfg, sit::solve_inv_tc_kernel, P, mapX, mapY32, mapY16));
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

}  // namespace rhqr
