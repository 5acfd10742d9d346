/*
 * rhqr.h -- C ABI of the GB300 (sm_103a) randomized Householder QR library.
 *
 * Method: L. Grigori, E. Timsit, "Randomized Householder QR" (2024).
 * A tall-skinny W (n x m, m << n) is factored as W = Q R with
 *   Q = (I_n - U T (Psi U)^t Psi) [I_m; 0]      (Thm. "mainthm", eq. generalcompact)
 * where Psi = diag(I_m, Omega) (eq. psi) and Omega is a k x (n-m) sketch
 * (Gaussian or SRHT, Section 2.3); Psi Q has orthonormal columns.
 *
 * Conventions of every entry point
 *  - Matrices are column-major with a leading dimension (ld >= rows).
 *  - All data pointers are DEVICE pointers owned by the caller, unless the
 *    comment says "host".  The library never frees them.
 *  - Small objects (Z = Psi X, S = Psi U, T, R) are float64.  High-dimensional
 *    objects (W, U, Q) are float64 or float32 (rhqr_dtype).
 *  - Work is enqueued on `stream`; a call returns before the GPU finishes.
 *    Argument errors are returned synchronously.  Conditions found on the GPU
 *    (breakdown, non-finite data, a bounded wait that ran out) are written to
 *    the caller's device `rhqr_info` and read after the stream synchronises.
 *  - No entry point traps, asserts or exits the process.
 *  - Indices (column numbers in rhqr_info) are 0-based.
 */
#ifndef RHQR_H
#define RHQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t (the default stream is NULL). */
typedef struct CUstream_st *rhqr_stream_t;

typedef enum {
  RHQR_OK = 0,
  RHQR_EINVAL = 1,      /* bad argument or shape                              */
  RHQR_ENOMEM = 2,      /* device allocation failed, or workspace too small    */
  RHQR_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed         */
  RHQR_EBREAKDOWN = 4,  /* rho = 0: a column's trailing part lies in Ker(Psi)  */
  RHQR_ENONFINITE = 5,  /* NaN or Inf met in the small FP64 computations       */
  RHQR_ETIMEOUT = 6,    /* a bounded device-side wait ran out                  */
  RHQR_ENOTSUP = 7      /* combination of options not implemented              */
} rhqr_status;

typedef enum { RHQR_SKETCH_GAUSSIAN = 0, RHQR_SKETCH_SRHT = 1 } rhqr_sketch_kind;
typedef enum { RHQR_F64 = 0, RHQR_F32 = 1, RHQR_BF16 = 2, RHQR_F16 = 3 } rhqr_dtype;
typedef enum { RHQR_ALG_LEFT = 0, RHQR_ALG_REC = 1, RHQR_ALG_BLOCK = 2 } rhqr_alg;

/* Opaque, library-owned sketch operator (device arrays inside). */
typedef struct rhqr_sketch_s *rhqr_sketch;

/* Device-resident result record, written by the kernels of one call. */
typedef struct {
  int32_t status;      /* rhqr_status of the device side                     */
  int32_t column;      /* column of a breakdown / non-finite value, else -1  */
  int32_t passes_done; /* recRHQR passes completed                           */
  int32_t reserved;
} rhqr_info;

/* Options of rhqr_factor.  rhqr_default_opts() fills the defaults. */
typedef struct {
  int32_t alg;          /* rhqr_alg (default RHQR_ALG_REC)                         */
  int32_t passes;       /* recRHQR passes, >= 1: pass i factors the Q of pass i-1
                           and R = R_p ... R_1 (default 1; ignored for LEFT)       */
  int32_t limbs_first;  /* 16-bit Gaussian sketch: X is split into this many
                           bf16/f16 limbs in pass 1 (1..3, default 2)              */
  int32_t limbs_refine; /* same for passes 2.. (1..3, default 2)                   */
  int32_t want_U;       /* write U (n x m, W's dtype); default 0                   */
  int32_t want_Q;       /* write the thin Q (n x m, W's dtype); default 1          */
  int32_t scaling;      /* reflector scaling of Algorithm 2: 0 = <u_j, e_j> = 1
                           (default), 1 = ||s_j|| = sqrt 2                         */
  int32_t solve;        /* float32 Q = X R^{-1} of recRHQR (m <= 256): 0 = tensor-core
                           product with the explicit inverse R^{-1} = D + E, Q = X D
                           + X E (default), 1 = tensor-core row-wise substitution  */
  int64_t wait_budget;  /* spin iterations of a device-side wait before it gives up
                           with RHQR_ETIMEOUT (0 = library default)                */
  int32_t block_size;   /* columns per block of RHQR_ALG_BLOCK (1..64, default 32) */
  int32_t column_scaling; /* recRHQR: 1 = equilibrate the columns of each pass's
                           sketch Z to unit norm before its Householder QR and
                           undo the scaling in R (default 0)                     */
} rhqr_opts;

/* Human-readable name of a status code (static string, never NULL). */
const char *rhqr_status_string(rhqr_status s);

/* Library version and the compute capability it was built for, e.g. 103. */
int32_t rhqr_version(void);
int32_t rhqr_built_arch(void);

void rhqr_default_opts(rhqr_opts *opts /* host */);

/*
 * rhqr_sketch_create -- draw the sketch Omega_full (k x n) from `seed`
 * (Section 2.3; the paper leaves the generator open, this library uses the
 * counter-based SplitMix64 scheme: entry i of stream t is the SplitMix64 output
 * function of seed * 0x9E3779B97F4A7C15 + t * 2^56 + i).
 *   kind = RHQR_SKETCH_SRHT: Omega_full = sqrt(N/k) P H D, N = 2^ceil(log2 n);
 *          stores N random signs and the k sampled rows (increasing).
 *   kind = RHQR_SKETCH_GAUSSIAN: Omega_full = G / sqrt(k), G i.i.d. N(0,1)
 *          (Box-Muller), materialised once in `omega_dtype` (F64, F32, BF16
 *          or F16) as a k x n row-major array (k*n elements of device memory);
 *          BF16 and F16 operators are stored a second time in the order the
 *          tensor-core sketch reads them (256 x 64 tiles, k and n rounded up),
 *          about twice the memory.
 * For a factorisation with m columns the sketch used is Psi_m = diag(I_m,
 * Omega) with Omega = columns m..n-1 of Omega_full (eq. psi).
 * Requires 1 <= k, k <= N (SRHT), n >= 2.  Allocates device memory (the only
 * allocating entry points are the *_create ones); the handle is immutable after
 * creation and may be used from several streams at once.  Synchronises
 * `stream` before returning.  *out is NULL on error.
 */
rhqr_status rhqr_sketch_create(int64_t n, int32_t k, int32_t kind, uint64_t seed,
                               int32_t omega_dtype, rhqr_stream_t stream, rhqr_sketch *out);

/* Frees the handle's device memory (NULL is accepted). */
rhqr_status rhqr_sketch_destroy(rhqr_sketch s);

/* Shape of a sketch (host outputs; any may be NULL). */
rhqr_status rhqr_sketch_shape(rhqr_sketch s, int64_t *n, int32_t *k, int32_t *kind,
                              int64_t *N, int32_t *omega_dtype);

/*
 * rhqr_sketch_export -- copy the drawn operator into caller device buffers:
 *   signs : N int8 values +1/-1 (SRHT only, else ignored; may be NULL)
 *   rows  : k int32 sampled rows, increasing (SRHT only; may be NULL)
 *   G     : k x n row-major Gaussian values in omega_dtype, ld = ldg >= n
 *           (Gaussian only; may be NULL)
 */
rhqr_status rhqr_sketch_export(rhqr_sketch s, int8_t *signs, int32_t *rows, void *G,
                               int64_t ldg, rhqr_stream_t stream);

/*
 * Workspace sizes (bytes) for rhqr_sketch_apply with c columns of dtype xt, and
 * for rhqr_factor / rhqr_reconstruct with an n x m matrix of dtype wt.
 */
rhqr_status rhqr_sketch_apply_workspace(rhqr_sketch s, int32_t m, int32_t xt, int64_t n,
                                        int32_t c, size_t *bytes);
rhqr_status rhqr_workspace_size(rhqr_sketch s, int64_t n, int32_t m, int32_t wt,
                                const rhqr_opts *opts, size_t *bytes);

/*
 * rhqr_sketch_apply -- Algorithm 1 (RHSketch): Z = Psi_m X = [X_{1:m}; Omega X_{m+1:n}].
 *   X : n x c, dtype xt (F64 or F32), leading dimension ldx >= n
 *   Z : (k+m) x c float64, leading dimension ldz >= k+m (output)
 * The top m rows are exact copies; the bottom k rows are the sketch.
 * Requires 0 <= m < n, m <= k.  There is no device status record: if a bounded
 * wait of the tensor-core kernel (float32 X, 16-bit Gaussian operator) runs
 * out, the bottom k rows of Z are NaN.
 */
rhqr_status rhqr_sketch_apply(rhqr_sketch s, int32_t m, const void *X, int32_t xt, int64_t n,
                              int32_t c, int64_t ldx, double *Z, int64_t ldz, void *ws,
                              size_t ws_bytes, rhqr_stream_t stream);

/*
 * rhqr_sketch_apply_rows -- one row shard's share of Algorithm 1 for a matrix
 * distributed by rows (each holder sketches its own rows, one sum of the
 * (k+m) x c results gives Z = Psi_m X; the paper's single synchronization):
 *   Z = Psi_m[:, row0 : row0+rows] X_local,
 * X_local (rows x c, dtype xt = F64 or F32, ldx >= rows) holding the global
 * rows row0 .. row0+rows-1 of an n-row X (n = the sketch's n).  The top block
 * of Z holds the shard's rows among the first m (zero elsewhere); the bottom k
 * rows the shard's columns of Omega applied to its rows >= m.  Gaussian: the
 * columns row0.. of Omega_full.  SRHT: the shard's segments of the Kronecker
 * split H_N = H_{N/N2} (x) H_{N2} transformed locally and combined with the
 * global segment signs; row0 must be a multiple of the segment length N2 =
 * min(N, 8192) (RHQR_EINVAL otherwise).  The float64 sums of the shards equal
 * rhqr_sketch_apply's Z to rounding.  ws: rhqr_sketch_apply_rows_workspace
 * bytes.  Requires 0 <= m <= k, m < n, 0 <= row0, row0 + rows <= n.
 */
rhqr_status rhqr_sketch_apply_rows_workspace(rhqr_sketch s, int32_t m, int32_t xt, int64_t row0, int64_t rows,
                                             int32_t c, size_t *bytes);
rhqr_status rhqr_sketch_apply_rows(rhqr_sketch s, int32_t m, const void *X, int32_t xt, int64_t row0, int64_t rows,
                                   int32_t c, int64_t ldx, double *Z, int64_t ldz, void *ws, size_t ws_bytes,
                                   rhqr_stream_t stream);

/*
 * rhqr_factor -- randomized Householder QR of W (n x m, dtype wt = F64 or F32).
 *  alg = RHQR_ALG_LEFT: Algorithm 4 (left-looking RHQR): column j is refreshed
 *        with the previous reflectors, w_j <- w_j - U T^t S^t Psi w_j, sketched,
 *        and its randomized Householder vector taken (Algorithm 2).
 *  alg = RHQR_ALG_BLOCK: Algorithm 5 (blockRHQR): the columns in blocks of
 *        opts->block_size; each block is first refreshed with every earlier
 *        block in turn (Y = Psi W_blk, W_blk <- W_blk - U_k T_k^t S_k^t Y, the
 *        block re-sketched each time), then factored by Algorithm 4 with its
 *        own reflectors.  T is returned as the compact-form T of all m
 *        reflectors (T^{-1} = sut(S^t S) + diag(1/beta), eq. generalwoodburry);
 *        its diagonal blocks are the blocks' T^(j) of Algorithm 5.
 *  alg = RHQR_ALG_REC : Algorithm 6 (recRHQR): Z = Psi W, Householder QR of Z
 *        gives S, T, R, and Q = W R^{-1} (equal to [I;0] - U T U_1^t, Section 3.3)
 *        is formed by a backward-stable row-wise triangular solve; with
 *        opts->passes = p > 1 the factorisation is repeated on its own Q and
 *        R = R_p ... R_1.  U (if wanted) solves W_2 = U_2 ut(T^t S^t Z) of the
 *        last pass (Algorithm 6, "backward solve").
 * Outputs (device):
 *   U  : n x m, dtype wt, ldu >= n   (required for LEFT and BLOCK, optional for REC)
 *   S  : (k+m) x m float64, lds >= k+m   (= Psi U of the representation)
 *   T  : m x m float64 (upper triangular, ld = m)
 *   R  : m x m float64 (upper triangular, ld = m)
 *   Q  : n x m, dtype wt, ldq >= n   (if opts->want_Q)
 *   info : device rhqr_info
 * ws/ws_bytes : device workspace of at least rhqr_workspace_size() bytes.
 * Requires m >= 1, n > m, k >= m, and for the Gaussian kind a sketch whose
 * stored n equals this n.  Breakdown (rho = 0) stops the factorisation and
 * reports the column in info.
 */
rhqr_status rhqr_factor(rhqr_sketch s, const void *W, int32_t wt, int64_t n, int32_t m,
                        int64_t ldw, const rhqr_opts *opts, void *U, int64_t ldu, double *S,
                        int64_t lds, double *T, double *R, void *Q, int64_t ldq, void *ws,
                        size_t ws_bytes, rhqr_info *info, rhqr_stream_t stream);

/*
 * rhqr_reconstruct -- the reconstruction steps of Algorithm 6: given the
 * Householder QR (S, T, R) of Z = Psi W (S with unit diagonal, Z = (I - S T
 * S^t)[R; 0]) and W itself, form M = ut(T^t S^t Z), U_1 = S_{1:m},
 * U_2 = W_2 M^{-1} (column recursion of Section 3.3) and, if Q != NULL,
 * Q = [I_m; 0] - U T U_1^t (Section 3.2).
 *   S (lds), Z (ldz): (k+m) x m float64; T, R: m x m float64 (ld = m)
 *   W: n x m dtype wt (ldw); U: n x m dtype wt (ldu); Q: n x m dtype wt or NULL
 */
rhqr_status rhqr_reconstruct(rhqr_sketch s, const double *S, int64_t lds, const double *T,
                             const double *R, const double *Z, int64_t ldz, const void *W,
                             int32_t wt, int64_t n, int32_t m, int64_t ldw, void *U, int64_t ldu,
                             void *Q, int64_t ldq, void *ws, size_t ws_bytes,
                             rhqr_stream_t stream);

/*
 * RHQR-Arnoldi (Algorithm 7): the Krylov basis of an operator A is kept in
 * compact form (U, S = Psi U, T) of mmax + 1 randomized reflectors, with
 * Psi = diag(I_{mmax+1}, Omega) (Omega = columns mmax+1..n-1 of the sketch).
 * The caller applies A: after begin(r0) gives q_1, every step(w = A q_j)
 * returns the Hessenberg column h_j and the next basis vector q_{j+1}, so that
 * A Q_m = Q_{m+1} H (eq. arnoldirelation) and Psi Q_{m+1} is orthonormal.
 *   create : n rows, up to mmax steps, basis dtype F64 or F32, reflector
 *            scaling 0 (unit diagonal) or 1 (||s|| = sqrt 2).  Allocates the
 *            handle's device memory (n x (mmax+1) basis plus small arrays).
 *            Requires mmax + 1 <= k and n > mmax + 1 (and n equal to the
 *            sketch's n for a Gaussian sketch).
 *   begin  : r0 = b - A x0 (n, device, basis dtype).  h0 (device, mmax + 1
 *            float64) receives (-sigma_1 rho_1, 0, ...); q1 (device, n) the
 *            first basis vector (may be NULL).
 *   step   : w = A q_j (device, n).  h (device, mmax + 1 float64) receives
 *            h_j; q_next (device, n, may be NULL) receives q_{j+1}.  At most
 *            mmax steps after begin; more return RHQR_EINVAL.
 *   export : copies U (n x (mmax+1), ldu), S ((k+mmax+1) x (mmax+1), lds),
 *            T ((mmax+1) x (mmax+1)) to caller device buffers (any may be
 *            NULL) and writes the number of reflectors taken to *count (host).
 * Breakdown (rho = 0) and non-finite values are reported in the device info.
 * Work is enqueued on `stream`; a handle serves one stream at a time.
 *
 * create_batch: nrhs independent processes (one per right-hand side, 1 ..
 * 65535) sharing the sketch; every kernel of begin, step and solution is
 * launched once for all of them.  The device arrays of the calls then hold
 * one column per process: r0, w, q1, q_next, x0, x are n x nrhs (ld n); h0, h
 * are (mmax+1) x nrhs (ld mmax+1); info holds nrhs records; export writes
 * nrhs stacked blocks (U + b ldu (mmax+1), S + b lds (mmax+1), T + b
 * (mmax+1)^2); solution reads H + b ldh mmax and writes y + b mmax, res + b.
 * rhqr_arnoldi_create is create_batch with nrhs = 1.
 */
typedef struct rhqr_arnoldi_s *rhqr_arnoldi;
rhqr_status rhqr_arnoldi_create(rhqr_sketch s, int64_t n, int32_t mmax, int32_t basis_dtype, int32_t scaling,
                                rhqr_arnoldi *out);
rhqr_status rhqr_arnoldi_create_batch(rhqr_sketch s, int64_t n, int32_t mmax, int32_t nrhs, int32_t basis_dtype,
                                      int32_t scaling, rhqr_arnoldi *out);
rhqr_status rhqr_arnoldi_destroy(rhqr_arnoldi a);
rhqr_status rhqr_arnoldi_begin(rhqr_arnoldi a, const void *r0, double *h0, void *q1, rhqr_info *info,
                               rhqr_stream_t stream);
rhqr_status rhqr_arnoldi_step(rhqr_arnoldi a, const void *w, double *h, void *q_next, rhqr_info *info,
                              rhqr_stream_t stream);
rhqr_status rhqr_arnoldi_export(rhqr_arnoldi a, void *U, int64_t ldu, double *S, int64_t lds, double *T,
                                int32_t *count, rhqr_stream_t stream);

/*
 * rhqr_arnoldi_solution -- the RHQR-GMRES update (Algorithm 8): after m steps
 * (1 <= m <= steps taken since begin), y = argmin || h0 - H y ||_2, which is
 * the sketched minimal-residual condition of eq. rgmresopti (Psi Q_{m+1} is
 * orthonormal, so || Psi (b - A x) || = || h0 - H y || for x = x0 + Q_m y),
 * and x = x0 + Q_m y with Q_m y = [y; 0] - U_m T_m S_m^t y (the compact form;
 * rows 0..m-1 of S's first m columns, the identity top block of Psi).
 *   H   : device float64, (m+1) x m (column j = the first m+1 entries of the
 *         h returned by step j), column-major, ldh >= m+1; read only.
 *   h0  : device float64, mmax+1 entries, as returned by begin.
 *   x0  : device, n, basis dtype (the x0 of r0 = b - A x0); x: device, n,
 *         basis dtype, may equal x0; x == NULL skips the update (y and res only).
 *   y   : device float64, m entries (output); res: device float64, 1 (output).
 * Float64 Givens rotations on the device; nothing is synchronised.  Returns
 * RHQR_EINVAL when m exceeds the steps taken or ldh < m+1.
 */
rhqr_status rhqr_arnoldi_solution(rhqr_arnoldi a, const double *H, int64_t ldh, int32_t m, const double *h0,
                                  const void *x0, void *x, double *y, double *res, rhqr_stream_t stream);
/* The same with x0 and x in dtype xdt (F64 or F32) independent of the basis
 * dtype: a float32 basis can update a float64 iterate (the restart residual
 * is then formed in float64, e.g. by rhqr_stencil_residual). */
rhqr_status rhqr_arnoldi_solution_x(rhqr_arnoldi a, const double *H, int64_t ldh, int32_t m, const double *h0,
                                    const void *x0, void *x, int32_t xdt, double *y, double *res,
                                    rhqr_stream_t stream);

/*
 * Batched recRHQR (Algorithm 6 with the refinement passes of rhqr_factor) of
 * `count` independent tall-skinny problems W_i (n_i x m_i) with SRHT sketches
 * s[i] (the paper factors one matrix; the batch runs many uneven ones at once).
 *   create : binds, once, the problems' sketches, shapes and device pointers
 *            (host arrays of `count` entries; every pointer they hold is a
 *            device pointer owned by the caller and must stay valid while the
 *            plan is used).  W_i: n_i x m_i, dtype wt (F64 or F32), ldw_i >=
 *            n_i; Q_i: n_i x m_i, dtype wt, ldq_i >= n_i (output, may alias
 *            nothing else); S_i: (k_i+m_i) x m_i float64, lds_i >= k_i+m_i;
 *            T_i, R_i: m_i x m_i float64 (ld = m_i).  opts: passes and scaling
 *            as for rhqr_factor (NULL = defaults; alg, limbs and want_* are
 *            ignored).  Requires 1 <= m_i <= 128, m_i < n_i <= N_i, m_i <= k_i
 *            and an SRHT sketch per problem.  Allocates the plan (a host
 *            object plus one device table) and synchronises the device.
 *   workspace_size : device workspace bytes of rhqr_factor_batched.
 *   rhqr_factor_batched : enqueues the whole batch on `stream` -- per pass one
 *            launch per phase covering every problem (SRHT stage A, stage B,
 *            FP64 Householder QR of each sketch, R accumulation, row solves
 *            Q = X R^{-1}), then one launch writing S, T (Woodbury form), R
 *            and the info records.  It allocates nothing, does not synchronise
 *            and launches a fixed sequence, so it may be captured into a CUDA
 *            graph and replayed as one graph launch while the bound pointers
 *            and the plan stay unchanged.  info: `count` device rhqr_info
 *            records, one per problem.  One plan serves one stream at a time.
 *   tune   : times the candidate launch shapes (stage-A threads, solve rows per
 *            block, solve grid cap) on the bound problems, `reps` launches
 *            each, keeps the fastest in the plan and writes them to choice
 *            (host, 3 int32; may be NULL).  It runs the batch first and
 *            overwrites the outputs; it synchronises the stream (do not
 *            capture it).  get/set_tuning read or restore a choice (set
 *            rejects values outside the candidate lists with RHQR_EINVAL).
 */
typedef struct rhqr_batch_s *rhqr_batch;
rhqr_status rhqr_batch_create(int32_t count, const rhqr_sketch *s, const void *const *W, int32_t wt,
                              const int64_t *n, const int32_t *m, const int64_t *ldw, const rhqr_opts *opts,
                              void *const *Q, const int64_t *ldq, double *const *S, const int64_t *lds,
                              double *const *T, double *const *R, rhqr_batch *out);
rhqr_status rhqr_batch_workspace_size(rhqr_batch b, size_t *bytes);
rhqr_status rhqr_batch_destroy(rhqr_batch b);
rhqr_status rhqr_factor_batched(rhqr_batch b, void *ws, size_t ws_bytes, rhqr_info *info, rhqr_stream_t stream);
rhqr_status rhqr_batch_tune(rhqr_batch b, void *ws, size_t ws_bytes, rhqr_info *info, int32_t reps,
                            int32_t *choice, rhqr_stream_t stream);
rhqr_status rhqr_batch_get_tuning(rhqr_batch b, int32_t *choice /* host, 3 */);
rhqr_status rhqr_batch_set_tuning(rhqr_batch b, const int32_t *choice /* host, 3 */);

/*
 * rhqr_blas2_rgs -- BLAS2-RGS (Algorithm 9, Section 6): the randomized
 * Householder QR of [0_m; W] written on W (n x m, dtype wt = F64 or F32, ldw),
 * with Omega = Omega_full of the sketch (k x n, no exact top block).  In exact
 * arithmetic it is randomized Gram-Schmidt: W = Q R with Omega Q orthonormal,
 * and T = I; in floating point T records the loss of sketched orthogonality.
 * Column j: z = Omega w_j, r = T^t S^t z, w = w_j - Q r, z = Omega w,
 * rho = ||z||, q_j = w / rho, s_j = z / rho, R[0:j, j] = r, R_jj = rho,
 * T[0:j, j] = -T S^t s_j, T_jj = 1.
 *   Q : n x m, dtype wt, ldq >= n (output);  R, T : m x m float64 (ld = m);
 *   S : k x m float64 (ld = k) = Omega Q;  info : device rhqr_info (a zero or
 *   non-finite rho is reported with its column).
 * ws/ws_bytes : device workspace of at least rhqr_blas2_rgs_workspace bytes.
 * Requires 1 <= m <= 1024, m <= k, n > m, and for the Gaussian kind n equal
 * to the sketch's n (else RHQR_EINVAL).
 */
rhqr_status rhqr_blas2_rgs_workspace(rhqr_sketch s, int32_t wt, int64_t n, int32_t m, size_t *bytes);
rhqr_status rhqr_blas2_rgs(rhqr_sketch s, const void *W, int32_t wt, int64_t n, int32_t m, int64_t ldw, void *Q,
                           int64_t ldq, double *R, double *T, double *S, void *ws, size_t ws_bytes, rhqr_info *info,
                           rhqr_stream_t stream);

/*
 * Operator of the RHQR-GMRES workload (not part of the method): the 2-D
 * convection-diffusion operator -Laplace(u) + pe (u_x + u_y) on the unit
 * square with zero Dirichlet boundary, g x g interior points (n = g^2, row
 * r = iy g + ix), h = 1/(g+1), central differences, scaled by h^2:
 *   (A u)_r = 4 u_r - (1 + c) u_{r-1} - (1 - c) u_{r+1} - (1 + c) u_{r-g}
 *             - (1 - c) u_{r+g},   c = pe h / 2  (neighbours off the grid are 0).
 * rhqr_stencil_apply: Y = A X for nrhs columns (X, Y: n x nrhs, ld n, dtype
 *   F64 or F32; Y must not overlap X).
 * rhqr_stencil_residual: R = B - A X formed in float64 and stored in dtype
 *   rdt (F64 or F32: the Krylov basis may be narrower than B and X), and
 *   norms[2b] = ||B[:, b] - A X[:, b]||_2, norms[2b+1] = ||B[:, b]||_2 of the
 *   float64 values (fixed-order sums) -- the restart residual of GMRES.
 *   work: rhqr_stencil_residual_workspace bytes.
 */
rhqr_status rhqr_stencil_apply(int32_t g, double pe, const void *X, int32_t dt, int32_t nrhs, void *Y,
                               rhqr_stream_t stream);
rhqr_status rhqr_stencil_residual_workspace(int32_t g, int32_t nrhs, size_t *bytes);
rhqr_status rhqr_stencil_residual(int32_t g, double pe, const void *B, const void *X, int32_t dt, int32_t nrhs, void *R,
                                  int32_t rdt, double *norms, void *work, size_t work_bytes, rhqr_stream_t stream);

/*
 * rhqr_trim_factor -- left-looking trimRHQR (Section 7): W (n x m, dtype wt =
 * F64 or F32) = H(u_1, Omega, 1) ... H(u_m, Omega, m) [R; 0] with the modified
 * randomized reflectors H(u, Omega, j) = I - beta u (Omega u)^t [0 Omega_{j:n}]
 * (eq. rhousebisbis), Omega = Omega_full of the sketch (k x n, no exact top
 * block).  The sketch size k may be smaller than m.  The method needs unit
 * first m columns of Omega: the SRHT has them; for a Gaussian sketch the first
 * m columns of Omega_full are normalised (Omega' = Omega_full with columns
 * 0..m-1 divided by their norms), and every sketch is taken with Omega'.
 * Column j is refreshed as w_j <- w_j - U Tt^t ut((Omega U)^t Omega) w_j
 * (eq. trimrhqrcompactfact), then trimRHVector takes u_j.
 * Outputs (device):
 *   U  : n x m, dtype wt, ldu >= n (unit diagonal, or ||Omega u_j|| = sqrt 2
 *        with scaling = 1)
 *   S  : k x m float64, lds >= k   (= Omega' U)
 *   T  : m x m float64 (right-wise products, eq. Tqdefbis):
 *        H_1 ... H_m = I - U T ut((Omega U)^t Omega)
 *   Tt : m x m float64 (left-wise products, eq. Sqdefbis):
 *        H_m ... H_1 = I - U Tt^t ut((Omega U)^t Omega)
 *   R  : m x m float64;  Q : n x m, dtype wt, ldq >= n, or NULL
 *        (Q = [I_m; 0] - U T ut(S^t Omega'_{:, 0:m}))
 *   info : device rhqr_info (breakdown: Omega' w' = 0)
 * ws/ws_bytes : device workspace of at least rhqr_trim_workspace bytes.
 * Requires 1 <= m <= 1024, n > m, and for the Gaussian kind n equal to the
 * sketch's n (else RHQR_EINVAL).
 */
rhqr_status rhqr_trim_workspace(rhqr_sketch s, int32_t wt, int64_t n, int32_t m, size_t *bytes);
rhqr_status rhqr_trim_factor(rhqr_sketch s, const void *W, int32_t wt, int64_t n, int32_t m, int64_t ldw,
                             int32_t scaling, void *U, int64_t ldu, double *S, int64_t lds, double *T, double *Tt,
                             double *R, void *Q, int64_t ldq, void *ws, size_t ws_bytes, rhqr_info *info,
                             rhqr_stream_t stream);

/*
 * Factorisation stream for matrices held in host memory (no counterpart in the
 * paper, which factors a matrix where the arithmetic runs).  Each submission
 * is one rhqr_factor (Algorithm 4 or 6, options as bound at create) of a host
 * W into host Q and R; the transfers of consecutive submissions overlap with
 * each other's factorisation.
 *   create : binds the sketch, W's dtype wt (F64 or F32), shape n x m and the
 *            options (NULL = defaults; want_Q must be 1), and allocates `depth`
 *            (1..4; 2 suffices for overlap) device buffer sets -- W, Q, U when
 *            needed, S, T, R, info and the rhqr_factor workspace each -- plus
 *            three non-blocking streams (copy in, compute, copy out).  The
 *            sketch must outlive the pipeline.
 *   submit : enqueues the copy of W (host, n x m column-major, ldw >= n) to a
 *            free buffer set, the factorisation, and the copies of Q (host,
 *            ldq >= n), R (host, m x m float64, ld = m) and, when not NULL, S
 *            (host, (k+m) x m float64, lds >= k+m), T (host, m x m) and info
 *            (host rhqr_info) back.  It returns once the work is enqueued: the
 *            host buffers must stay valid and unchanged (W) or unread (outputs)
 *            until rhqr_pipeline_wait returns.  Page-locked host buffers
 *            (cudaHostAlloc / cudaHostRegister) are needed for the copies to
 *            overlap; pageable ones give the same results, serialised.
 *            Argument errors of the factorisation are returned here.
 *   wait   : blocks until every submitted factorisation's outputs are in host
 *            memory; a device-side status (breakdown, non-finite) is in info.
 *   destroy: waits, then frees the buffers, streams and events.
 * One pipeline is driven by one host thread at a time.
 */
typedef struct rhqr_pipeline_s *rhqr_pipeline;
rhqr_status rhqr_pipeline_create(rhqr_sketch s, int32_t wt, int64_t n, int32_t m, const rhqr_opts *opts,
                                 int32_t depth, rhqr_pipeline *out);
rhqr_status rhqr_pipeline_submit(rhqr_pipeline p, const void *W, int64_t ldw, void *Q, int64_t ldq, double *R,
                                 double *S, int64_t lds, double *T, rhqr_info *info);
rhqr_status rhqr_pipeline_wait(rhqr_pipeline p);
rhqr_status rhqr_pipeline_destroy(rhqr_pipeline p);

/*
 * rhqr_sketch_apply_noalloc -- rhqr_sketch_apply without a caller workspace;
 * the paper has no counterpart.  For callers that cannot allocate device
 * memory when they call: framework hooks and custom operators whose rules
 * forbid device allocation at call time, real-time paths that must not block
 * on cudaMalloc, and host applications that own all device memory and cannot
 * hand the library a workspace.  Arguments as for rhqr_sketch_apply (X and Z
 * are still the caller's).
 * Scratch: a fixed RHQR_NOALLOC_SCRATCH_BYTES device array inside the library
 * that every GPU loading the library holds until the process exits; a call
 * needing more scratch (large k * c) returns RHQR_ENOMEM and does nothing.
 * The call allocates nothing.  Its first call on a device looks up the
 * array's device address (with that device current) and caches it with the
 * device's current CUDA context; a call from another context of the device
 * (after cudaDeviceReset, for instance) looks it up again.  Make that first
 * call before any stream capture.  All calls share the array, which keeps the
 * last call's contents; calls whose work overlaps on the GPU (several streams
 * or threads) race on it and must be serialised by the caller.
 */
#define RHQR_NOALLOC_SCRATCH_BYTES (24u * 1024u * 1024u)
rhqr_status rhqr_sketch_apply_noalloc(rhqr_sketch s, int32_t m, const void *X, int32_t xt, int64_t n, int32_t c,
                                      int64_t ldx, double *Z, int64_t ldz, rhqr_stream_t stream);

/*
 * Instrumentation (no counterpart in the paper).
 * rhqr_launch_count: number of kernels this library has launched so far in the
 *   process (every launch site counts itself; host-side counter).
 * rhqr_profile_enable(1): reset the phase timers and start recording a pair of
 *   CUDA events around each phase on the stream the phase is launched on;
 *   (0) stops recording.  rhqr_profile_read copies, for phase i < n, the summed
 *   event time in milliseconds and the number of timed calls, synchronising on
 *   the recorded events; returns the number of phases.  Phases: 0 sketch
 *   (Algorithm 1), 1 Householder QR of the sketch, 2 T factor, 3 row solves /
 *   Q formation, 4 other small FP64 work, 5 left-looking column steps.
 */
int64_t rhqr_launch_count(void);

/*
 * rhqr_last_cuda_error: the CUDA runtime error code (cudaError_t value) of the
 * most recent call of this library that returned RHQR_ECUDA, 0 if none did;
 * process-wide, not per thread.  rhqr_cuda_error_name: its name (a static
 * string owned by the CUDA runtime, e.g. "cudaErrorInvalidClusterSize").
 */
int32_t rhqr_last_cuda_error(void);
const char *rhqr_cuda_error_name(int32_t code);
void rhqr_profile_enable(int32_t on);
int32_t rhqr_profile_read(double *ms /* host, n */, int64_t *calls /* host, n */, int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* RHQR_H */
