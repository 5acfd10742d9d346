// Blocked Householder QR of the sketch Z (p x m, float64) for recRHQR
// (Algorithm 6), same conventions as the column-by-column version in small.cu
// (Algorithm 2 with Psi = I: sigma = sign(z_jj) with sign(0) = +1, rho =
// ||z_{j:}||, v = z_{j:} / gamma with v_j = 1 or the ||v|| = sqrt 2 scaling,
// beta = 1 + |z_jj| / rho, r_jj = -sigma rho).
//
// Panels of 32 columns.  A panel is factored by one cluster of CTAs that hold
// its rows in shared memory; each column costs one cluster barrier, and the
// partial sums of the CTAs are pushed into each other's shared memory and
// added in a fixed order, so the result does not depend on timing.  The one
// reduction per column takes the dots of the unscaled column z_j with every
// panel column (its own: ||z_{j:}||^2) and, with row j of the panel pushed by
// its owner, yields rho and every product the column needs: with
// v_j(i) = rdiv z_j(i) below the diagonal and v_j(j) = vjj,
//   v_j . y = vjj y(j) + rdiv (z_j . y - z_jj y(j))   (rows >= j)
// for y = z_c (c > j) and y = v_k (k < j).  The
// panel's reflectors are then applied to the trailing columns in compact form,
// Z_t <- (I - V T^t V^t) Z_t, one CTA per trailing column.  T (upper
// triangular, T_jj = beta_j) is never formed: T^{-1} = diag(1/beta) +
// striu(V^t V), the panel collects V^t V with its own dot products, and the
// update finds T^t (V^t z) by forward substitution with T^{-t}.
#include <algorithm>

#include "common.cuh"
#include "small.cuh"
#include "tcgen05.cuh"

namespace rhqr {
namespace hb {

__device__ __forceinline__ int64_t clamp64(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

constexpr int NB = 32;       // panel width
constexpr int PT = 256;      // threads of a panel CTA
constexpr int UT = 256;      // threads of an update CTA
constexpr size_t SMEM_MAX = 200 * 1024;
constexpr int MAXCS = 16;    // largest cluster

struct Args {
  double *A;  // p x m working copy, ld = p
  int64_t p;
  int32_t m, j0, nbp, per;  // panel [j0, j0 + nbp); rows per CTA of the panel cluster
  double *S;
  int64_t lds;
  double *beta, *rdiag, *Tp;  // beta (m), -sigma rho (m), panel T (NB x NB, ld NB)
  int *bad;                   // set once a breakdown / non-finite value is met
  rhqr_info *info;
  int32_t scaling;
};

__global__ void __launch_bounds__(PT) hqr_panel_kernel(Args a) {
  extern __shared__ __align__(16) double sm[];
  __shared__ double sh[4];
  if (*(volatile int *)a.bad) return;  // identical for every CTA of the cluster
  const uint32_t rank = tc::cluster_ctarank(), cs = gridDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = a.per, nbp = a.nbp, j0 = a.j0;
  const int64_t p = a.p;
  const int64_t row0 = (int64_t)j0 + (int64_t)rank * per;
  const int nloc = (int)clamp64(p - row0, 0, per);
  const int ps = per | 1;  // odd column stride: lanes reading one row of 32 columns hit distinct banks
  double *pan = sm;                      // [NB][ps]: column c, local row i
  // part and zrow are double-buffered by column parity: a CTA pushes column
  // j + 1's values while a slower peer may still be summing column j's (one
  // cluster barrier per column), and it cannot reach column j + 2's push
  // before that peer has passed column j + 1's barrier.
  double *part0 = sm + NB * ps;           // [2][MAXCS][NB + 1]: partial sums pushed by every CTA
  double *gram = part0 + 2 * MAXCS * (NB + 1);  // [NB][NB]: gram[k * NB + l] = v_k . v_l (k < l), whole cluster
  double *wsh = gram + NB * NB;          // [NB]: beta (v_j . z_c)
  double *zrow0 = wsh + NB;              // [2][NB]: row j of the panel, pushed by its owner
  double *dsum = zrow0 + 2 * NB;         // [NB]: z_j . (column c), rows >= j, whole cluster
  double *red = dsum + NB;               // [PT / 32][32]: per-warp partial dots
  for (int e = tid; e < nbp * per; e += PT) {
    const int c = e / per, i = e % per;
    pan[c * ps + i] = i < nloc ? a.A[(int64_t)(j0 + c) * p + row0 + i] : 0.0;
  }
  __syncthreads();
  tc::cluster_sync();  // every CTA of the cluster runs before any pushes into its shared memory
  for (int jc = 0; jc < nbp; ++jc) {
    const int64_t j = (int64_t)j0 + jc;
    const int lo = (int)clamp64(j - row0, 0, nloc);  // first own row >= j
    const uint32_t owner = (uint32_t)(jc / per);
    double *part = part0 + (jc & 1) * MAXCS * (NB + 1);
    double *zrow = zrow0 + (jc & 1) * NB;
    // ---- partial dots z_j . (column c) over this CTA's rows >= j, lane =
    //      column (c = jc gives ||z_{j:}||^2), warp = every 8th own row: no
    //      butterfly reductions (FP64 instructions are the scarce resource); the
    //      8 warp partials of a column are added by a fixed tree and pushed to
    //      every CTA, with row j of the panel from its owner.
    {
      double d = 0.0;
      if (lane < nbp)
        for (int i = lo + warp; i < nloc; i += PT / 32) d += pan[jc * ps + i] * pan[lane * ps + i];
      red[warp * 32 + lane] = d;
    }
    __syncthreads();
    if (warp == 0 && lane < nbp) {
      const double *rw = red + lane;
      const double d = ((rw[0] + rw[32]) + (rw[64] + rw[96])) + ((rw[128] + rw[160]) + (rw[192] + rw[224]));
      const double zr = rank == owner ? pan[lane * ps + (jc - (int)owner * per)] : 0.0;
      for (uint32_t r = 0; r < cs; ++r) {
        tc::st_cluster_f64(tc::map_to_rank(part + rank * (NB + 1) + lane, r), d);
        if (rank == owner) tc::st_cluster_f64(tc::map_to_rank(zrow + lane, r), zr);
      }
    }
    tc::cluster_sync();
    // sums over ranks, lane = column, by a fixed tree over the 16 (or fewer) ranks
    if (warp == 0 && lane < nbp) {
      double v[MAXCS];
#pragma unroll
      for (int r = 0; r < MAXCS; ++r) v[r] = r < (int)cs ? part[r * (NB + 1) + lane] : 0.0;
#pragma unroll
      for (int h = MAXCS / 2; h > 0; h >>= 1)
#pragma unroll
        for (int r = 0; r < h; ++r) v[r] = v[2 * r] + v[2 * r + 1];
      dsum[lane] = v[0];
    }
    __syncthreads();
    if (tid == 0) {
      // one reciprocal square root and one division per column (FP64 square
      // roots and divisions are long dependent sequences on this GPU)
      const double tot = dsum[jc];
      const double zjj = zrow[jc];
      const bool zero = tot == 0.0;
      const double rinv = rsqrt(tot);  // 1 / rho
      const double rho = tot * rinv;
      const bool fail = zero || !isfinite(rho) || !isfinite(zjj);
      if (fail) {
        if (rank == 0) {
          set_status(a.info, zero ? RHQR_EBREAKDOWN : RHQR_ENONFINITE, (int32_t)j);
          *a.bad = 1;
        }
      } else {
        const double sigma = zjj < 0.0 ? -1.0 : 1.0;
        const double gamma = zjj + sigma * rho;
        if (a.scaling == 0) {  // v_j = 1, beta = 1 + |z_jj| / rho
          sh[0] = 1.0 + fabs(zjj) * rinv;
          sh[1] = 1.0 / gamma;
          sh[2] = 1.0;
        } else {               // ||v|| = sqrt 2, beta = 1
          const double rdiv = rsqrt(rho * (rho + fabs(zjj)));
          sh[0] = 1.0;
          sh[1] = rdiv;
          sh[2] = gamma * rdiv;
        }
        if (rank == 0) {
          a.beta[j] = sh[0];
          a.rdiag[j] = -sigma * rho;
        }
      }
      sh[3] = fail ? 1.0 : 0.0;
    }
    __syncthreads();
    if (sh[3] != 0.0) {
      tc::cluster_sync();  // no CTA leaves while another may still read its shared memory
      return;
    }
    const double beta = sh[0], rdiv = sh[1], vjj = sh[2];
    // w_c = beta (v_j . z_c) for c > j; column j of the panel's V^t V for k < j
    if (warp == 0 && lane < nbp && lane != jc) {
      const double zjj = zrow[jc], y = zrow[lane];
      const double vy = vjj * y + rdiv * (dsum[lane] - zjj * y);
      if (lane > jc) wsh[lane] = beta * vy;
      else gram[lane * NB + jc] = vy;
    }
    for (int i = lo + tid; i < nloc; i += PT) {
      const int64_t gi = row0 + i;
      pan[jc * ps + i] = gi == j ? vjj : pan[jc * ps + i] * rdiv;
    }
    __syncthreads();
    for (int e = tid; e < (nbp - jc - 1) * (nloc - lo); e += PT) {
      const int c = jc + 1 + e / (nloc - lo), i = lo + e % (nloc - lo);
      pan[c * ps + i] -= pan[jc * ps + i] * wsh[c];
    }
    __syncthreads();
  }
  // write the factored panel back: A (v below the diagonal, R above), S
  for (int e = tid; e < nbp * nloc; e += PT) {
    const int c = e / nloc, i = e % nloc;
    const int64_t gi = row0 + i, j = (int64_t)j0 + c;
    const double v = pan[c * ps + i];
    a.A[j * p + gi] = v;
    a.S[j * a.lds + gi] = gi < j ? 0.0 : v;
  }
  if (rank == 0)
    for (int e = tid; e < nbp * j0; e += PT) a.S[(int64_t)(j0 + e / j0) * a.lds + e % j0] = 0.0;
  // The panel's T is not formed: with T^{-1} = diag(1/beta) + striu(V^t V) the
  // trailing update solves with it instead (one warp per update CTA), so the
  // panel only hands over V^t V (strict upper part, column-major NB x NB).
  if (rank == 0)
    for (int e = tid; e < nbp * NB; e += PT) {
      const int k = e % NB, l = e / NB;
      a.Tp[e] = k < l ? gram[k * NB + l] : 0.0;
    }
  tc::cluster_sync();  // peers finish reading this CTA's shared memory
}

// Z[:, c] <- Z[:, c] - V T^t V^t Z[:, c] for one trailing column c per CTA,
// with T^t w found by forward substitution in T^{-t} = diag(1/beta) +
// striu(V^t V)^t (Tp holds the panel's V^t V, column l = entries (k, l), k < l)
__global__ void __launch_bounds__(UT) hqr_update_kernel(Args a) {
  __shared__ double w[NB], w2[NB], gsh[NB * NB];
  if (*(volatile int *)a.bad) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t p = a.p, j0 = a.j0;
  const int nbp = a.nbp;
  double *z = a.A + (int64_t)(j0 + nbp + blockIdx.x) * p;
  for (int e = tid; e < nbp * NB; e += UT) gsh[e] = a.Tp[e];
  // w_k = v_k . z: warp w takes k = w, w + 8, w + 16, w + 24 together (four
  // independent FMA chains per lane, z read once for all four); V = S is zero
  // above each reflector's diagonal, so every k starts at row j0
  static_assert(UT / 32 * 4 == NB, "four reflectors per warp");
  {
    const int k0 = warp, k1 = warp + 8, k2 = warp + 16, k3 = warp + 24;
    const double *v0 = a.S + (j0 + (k0 < nbp ? k0 : 0)) * a.lds, *v1 = a.S + (j0 + (k1 < nbp ? k1 : 0)) * a.lds;
    const double *v2 = a.S + (j0 + (k2 < nbp ? k2 : 0)) * a.lds, *v3 = a.S + (j0 + (k3 < nbp ? k3 : 0)) * a.lds;
    double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
    for (int64_t i = j0 + lane; i < p; i += 32) {
      const double zi = z[i];
      if (k0 < nbp) d0 += v0[i] * zi;
      if (k1 < nbp) d1 += v1[i] * zi;
      if (k2 < nbp) d2 += v2[i] * zi;
      if (k3 < nbp) d3 += v3[i] * zi;
    }
    d0 = warp_sum(d0);
    d1 = warp_sum(d1);
    d2 = warp_sum(d2);
    d3 = warp_sum(d3);
    if (lane == 0) {
      if (k0 < nbp) w[k0] = d0;
      if (k1 < nbp) w[k1] = d1;
      if (k2 < nbp) w[k2] = d2;
      if (k3 < nbp) w[k3] = d3;
    }
  }
  __syncthreads();
  if (warp == 0) {
    // w2_q = beta_q (w_q - sum_{k<q} G_kq w2_k); lane i keeps its running sum
    const double bi = lane < nbp ? a.beta[j0 + lane] : 0.0;
    const double wi = lane < nbp ? w[lane] : 0.0;
    double s = 0.0, res = 0.0;
    for (int q = 0; q < nbp; ++q) {
      const double t = __shfl_sync(0xffffffffu, bi * (wi - s), q);
      if (lane == q) res = t;
      if (lane > q && lane < nbp) s += gsh[lane * NB + q] * t;
    }
    if (lane < nbp) w2[lane] = res;
  }
  __syncthreads();
  // z_i -= sum_k v_k(i) w2_k (zeros above the diagonals included), four chains
  for (int64_t i = j0 + tid; i < p; i += UT) {
    const double *vi = a.S + j0 * a.lds + i;
    double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0;
    int k = 0;
    for (; k + 3 < nbp; k += 4) {
      c0 += vi[(int64_t)k * a.lds] * w2[k];
      c1 += vi[(int64_t)(k + 1) * a.lds] * w2[k + 1];
      c2 += vi[(int64_t)(k + 2) * a.lds] * w2[k + 2];
      c3 += vi[(int64_t)(k + 3) * a.lds] * w2[k + 3];
    }
    for (; k < nbp; ++k) c0 += vi[(int64_t)k * a.lds] * w2[k];
    z[i] -= (c0 + c1) + (c2 + c3);
  }
}

// R (m x m): the strict upper part from Z, the diagonal -sigma rho
__global__ void hqr_r_kernel(const double *A, int64_t p, int32_t m, const double *rdiag, const int *bad, double *R) {
  if (*bad) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)m * m) return;
  const int j = (int)(idx / m), i = (int)(idx % m);
  R[idx] = i < j ? A[(int64_t)j * p + i] : (i == j ? rdiag[j] : 0.0);
}

static size_t panel_smem(int per) {
  return sizeof(double) * ((size_t)NB * (per | 1) + 2 * (size_t)MAXCS * (NB + 1) + (size_t)NB * NB + 4 * NB + (size_t)PT);
}

// Largest cluster (16, 8 or 4 CTAs) that fits the first panel of p rows.
static int cluster_size(int64_t p) {
  static int64_t cached_p = -1;
  static int cached = 0;
  if (cached_p == p) return cached;
  int best = 0;
  for (int cs : {16, 8, 4}) {
    const size_t smem = panel_smem((int)ceil_div(p, cs));
    if (smem > SMEM_MAX) continue;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(PT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, hqr_panel_kernel, &cfg) == cudaSuccess && n >= 1) {
      best = cs;
      break;
    }
    (void)cudaGetLastError();
  }
  cached_p = p;
  cached = best;
  return best;
}

}  // namespace hb

size_t hqr_blocked_workspace_bytes(int64_t p, int32_t m) {
  Carver c(nullptr, 0);
  c.take<double>((size_t)p * m);
  c.take<double>((size_t)m);
  c.take<double>((size_t)hb::NB * hb::NB);
  c.take<int>(4);
  return c.used() + 256;
}

rhqr_status householder_qr_blocked(const double *Z, int64_t ldz, int64_t p, int32_t m, double *S, int64_t lds,
                                   double *R, double *beta, int32_t scaling, void *ws, size_t ws_bytes,
                                   rhqr_info *info, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    RHQR_CUDA_TRY(cudaFuncSetAttribute(hb::hqr_panel_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    RHQR_CUDA_TRY(
        cudaFuncSetAttribute(hb::hqr_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hb::SMEM_MAX));
    attr_set = true;
  }
  const int cs = hb::cluster_size(p);
  if (cs == 0) return RHQR_ENOTSUP;
  Carver c(ws, ws_bytes);
  double *A = c.take<double>((size_t)p * m);
  double *rdiag = c.take<double>((size_t)m);
  double *Tp = c.take<double>((size_t)hb::NB * hb::NB);
  int *bad = c.take<int>(4);
  if (c.overflow()) return RHQR_ENOMEM;
  RHQR_TRY(copy_f64_2d(Z, ldz, p, m, A, p, st));
  RHQR_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), st));
  hb::Args a{A, p, m, 0, 0, 0, S, lds, beta, rdiag, Tp, bad, info, scaling};
  for (int j0 = 0; j0 < m; j0 += hb::NB) {
    a.j0 = j0;
    a.nbp = std::min(hb::NB, m - j0);
    a.per = (int)ceil_div(p - j0, cs);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cs, 1, 1);
    cfg.blockDim = dim3(hb::PT, 1, 1);
    cfg.dynamicSmemBytes = hb::panel_smem(a.per);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    RHQR_CUDA_TRY(cudaLaunchKernelEx(&cfg, hb::hqr_panel_kernel, a));
    RHQR_LAUNCH_CHECK();
    const int nt = m - j0 - a.nbp;
    if (nt > 0) {
      hb::hqr_update_kernel<<<nt, hb::UT, 0, st>>>(a);
      RHQR_LAUNCH_CHECK();
    }
  }
  hb::hqr_r_kernel<<<(unsigned)ceil_div((int64_t)m * m, 256), 256, 0, st>>>(A, p, m, rdiag, bad, R);
  RHQR_LAUNCH_CHECK();
  return RHQR_OK;
}

}  // namespace rhqr
