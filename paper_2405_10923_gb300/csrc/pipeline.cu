// Factorisation stream for host-resident matrices (rhqr_pipeline_* in rhqr.h).
//
// The paper factors one matrix held where the arithmetic runs; a user whose
// matrices live in host memory pays the transfers of W in and Q out, which on
// this GPU move more bytes than the factorisation itself reads at HBM speed.
// The pipeline hides them behind the arithmetic: it owns `depth` device buffer
// sets and three streams, and submission i
//   copy-in stream : waits until set i % depth is no longer read by the
//                    factorisation that last used it, copies W_i host -> device
//   compute stream : waits for that copy and for the copy-out of the set's
//                    previous outputs, runs rhqr_factor on the set
//   copy-out stream: waits for the factorisation, copies Q_i, R_i (and S_i,
//                    T_i, info_i when asked) device -> host
// so the copy of W_{i+1} and of Q_{i-1} run while W_i is factored.  All
// ordering is by CUDA events; submit only enqueues.
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

struct rhqr_pipeline_s {
  struct Slot {
    void *W = nullptr, *Q = nullptr, *U = nullptr;
    double *S = nullptr, *T = nullptr, *R = nullptr;
    rhqr_info *info = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    cudaEvent_t in_done = nullptr, comp_done = nullptr, out_done = nullptr;
  };
  rhqr_sketch s = nullptr;
  int32_t wt = 0, m = 0, k = 0;
  int64_t n = 0;
  rhqr_opts o{};
  std::vector<Slot> slots;
  cudaStream_t s_in = nullptr, s_comp = nullptr, s_out = nullptr;
  void *mem = nullptr;
  int64_t submitted = 0;
};

namespace rhqr {

static size_t elem_size(int32_t wt) { return wt == RHQR_F64 ? 8 : 4; }

// Byte layout of one slot; with base == nullptr only the size is computed.
// Device copies of W, Q and U use ld = n rounded up to 32 elements, so that
// every column starts on a 128-byte boundary (the tensor-memory-access copies
// of the float32 sketch and solve need 16-byte aligned strides).
static int64_t device_ld(int64_t n) { return (n + 31) / 32 * 32; }

static bool carve_slot(Carver &c, int64_t n, int32_t m, int32_t k, int32_t wt, bool want_U, size_t ws_bytes,
                       rhqr_pipeline_s::Slot &sl) {
  const size_t es = elem_size(wt);
  const int64_t p = (int64_t)k + m, ld = device_ld(n);
  sl.W = c.take<char>((size_t)ld * m * es);
  sl.Q = c.take<char>((size_t)ld * m * es);
  sl.U = want_U ? c.take<char>((size_t)ld * m * es) : nullptr;
  sl.S = c.take<double>((size_t)p * m);
  sl.T = c.take<double>((size_t)m * m);
  sl.R = c.take<double>((size_t)m * m);
  sl.info = c.take<rhqr_info>(1);
  sl.ws = c.take<char>(ws_bytes);
  sl.ws_bytes = ws_bytes;
  return !c.overflow();
}

static void release(rhqr_pipeline_s *p) {
  for (auto &sl : p->slots) {
    if (sl.in_done) cudaEventDestroy(sl.in_done);
    if (sl.comp_done) cudaEventDestroy(sl.comp_done);
    if (sl.out_done) cudaEventDestroy(sl.out_done);
  }
  if (p->s_in) cudaStreamDestroy(p->s_in);
  if (p->s_comp) cudaStreamDestroy(p->s_comp);
  if (p->s_out) cudaStreamDestroy(p->s_out);
  if (p->mem) cudaFree(p->mem);
  delete p;
}

}  // namespace rhqr

using namespace rhqr;

extern "C" {

rhqr_status rhqr_pipeline_create(rhqr_sketch s, int32_t wt, int64_t n, int32_t m, const rhqr_opts *opts,
                                 int32_t depth, rhqr_pipeline *out) {
  if (out == nullptr) return RHQR_EINVAL;
  *out = nullptr;
  if (s == nullptr || (wt != RHQR_F64 && wt != RHQR_F32) || m < 1 || n <= m || depth < 1 || depth > 4)
    return RHQR_EINVAL;
  rhqr_opts o;
  if (opts) o = *opts;
  else rhqr_default_opts(&o);
  if (!o.want_Q) return RHQR_EINVAL;  // the pipeline exists to deliver Q to the host
  int64_t sn = 0, sN = 0;
  int32_t sk = 0, skind = 0, sdt = 0;
  RHQR_TRY(rhqr_sketch_shape(s, &sn, &sk, &skind, &sN, &sdt));
  if (sk < m) return RHQR_EINVAL;
  size_t ws_bytes = 0;
  RHQR_TRY(rhqr_workspace_size(s, n, m, wt, &o, &ws_bytes));
  const bool want_U = o.want_U || o.alg != RHQR_ALG_REC;

  rhqr_pipeline_s *p = new (std::nothrow) rhqr_pipeline_s();
  if (p == nullptr) return RHQR_ENOMEM;
  p->s = s;
  p->wt = wt;
  p->n = n;
  p->m = m;
  p->k = sk;
  p->o = o;
  p->slots.resize((size_t)depth);
  size_t slot_bytes = 0;
  {
    Carver c(nullptr, 0);
    rhqr_pipeline_s::Slot tmp;
    carve_slot(c, n, m, sk, wt, want_U, ws_bytes, tmp);
    slot_bytes = align_up(c.used(), 256);
  }
  if (cudaMalloc(&p->mem, slot_bytes * (size_t)depth) != cudaSuccess) {
    (void)cudaGetLastError();
    p->mem = nullptr;
    release(p);
    return RHQR_ENOMEM;
  }
  bool ok = cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&p->s_comp, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking) == cudaSuccess;
  for (int32_t i = 0; ok && i < depth; ++i) {
    auto &sl = p->slots[(size_t)i];
    Carver c((char *)p->mem + slot_bytes * (size_t)i, slot_bytes);
    ok = carve_slot(c, n, m, sk, wt, want_U, ws_bytes, sl) &&
         cudaEventCreateWithFlags(&sl.in_done, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&sl.comp_done, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&sl.out_done, cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    (void)cudaGetLastError();
    release(p);
    return RHQR_ECUDA;
  }
  *out = p;
  return RHQR_OK;
}

// Column-major block copy (rows x cols, element size es): one contiguous copy
// when both leading dimensions equal the column length, else a pitched copy.
static cudaError_t copy_cols(void *dst, int64_t dld, const void *src, int64_t sld, int64_t rows, int64_t cols,
                             size_t es, cudaMemcpyKind kind, cudaStream_t st) {
  if (dld == rows && sld == rows) return cudaMemcpyAsync(dst, src, (size_t)rows * (size_t)cols * es, kind, st);
  return cudaMemcpy2DAsync(dst, (size_t)dld * es, src, (size_t)sld * es, (size_t)rows * es, (size_t)cols, kind, st);
}

rhqr_status rhqr_pipeline_submit(rhqr_pipeline p, const void *W, int64_t ldw, void *Q, int64_t ldq, double *R,
                                 double *S, int64_t lds, double *T, rhqr_info *info) {
  if (p == nullptr || W == nullptr || Q == nullptr || R == nullptr) return RHQR_EINVAL;
  const int64_t n = p->n, pk = (int64_t)p->k + p->m, ld = device_ld(n);
  const int32_t m = p->m;
  if (ldw < n || ldq < n || (S != nullptr && lds < pk)) return RHQR_EINVAL;
  const size_t es = elem_size(p->wt);
  auto &sl = p->slots[(size_t)(p->submitted % (int64_t)p->slots.size())];

  // W in: the slot's previous factorisation must have finished reading W
  RHQR_CUDA_TRY(cudaStreamWaitEvent(p->s_in, sl.comp_done, 0));
  RHQR_CUDA_TRY(copy_cols(sl.W, ld, W, ldw, n, m, es, cudaMemcpyHostToDevice, p->s_in));
  RHQR_CUDA_TRY(cudaEventRecord(sl.in_done, p->s_in));

  // factorisation: after W arrived and after the previous outputs left
  RHQR_CUDA_TRY(cudaStreamWaitEvent(p->s_comp, sl.in_done, 0));
  RHQR_CUDA_TRY(cudaStreamWaitEvent(p->s_comp, sl.out_done, 0));
  RHQR_TRY(rhqr_factor(p->s, sl.W, p->wt, n, m, ld, &p->o, sl.U, ld, sl.S, pk, sl.T, sl.R, sl.Q, ld, sl.ws, sl.ws_bytes,
                       sl.info, (rhqr_stream_t)p->s_comp));
  RHQR_CUDA_TRY(cudaEventRecord(sl.comp_done, p->s_comp));

  // outputs out
  RHQR_CUDA_TRY(cudaStreamWaitEvent(p->s_out, sl.comp_done, 0));
  RHQR_CUDA_TRY(copy_cols(Q, ldq, sl.Q, ld, n, m, es, cudaMemcpyDeviceToHost, p->s_out));
  RHQR_CUDA_TRY(cudaMemcpyAsync(R, sl.R, sizeof(double) * (size_t)m * m, cudaMemcpyDeviceToHost, p->s_out));
  if (S != nullptr)
    RHQR_CUDA_TRY(cudaMemcpy2DAsync(S, (size_t)lds * 8, sl.S, (size_t)pk * 8, (size_t)pk * 8, (size_t)m,
                                    cudaMemcpyDeviceToHost, p->s_out));
  if (T != nullptr)
    RHQR_CUDA_TRY(cudaMemcpyAsync(T, sl.T, sizeof(double) * (size_t)m * m, cudaMemcpyDeviceToHost, p->s_out));
  if (info != nullptr)
    RHQR_CUDA_TRY(cudaMemcpyAsync(info, sl.info, sizeof(rhqr_info), cudaMemcpyDeviceToHost, p->s_out));
  RHQR_CUDA_TRY(cudaEventRecord(sl.out_done, p->s_out));
  ++p->submitted;
  return RHQR_OK;
}

rhqr_status rhqr_pipeline_wait(rhqr_pipeline p) {
  if (p == nullptr) return RHQR_EINVAL;
  RHQR_CUDA_TRY(cudaStreamSynchronize(p->s_in));
  RHQR_CUDA_TRY(cudaStreamSynchronize(p->s_comp));
  RHQR_CUDA_TRY(cudaStreamSynchronize(p->s_out));
  return RHQR_OK;
}

rhqr_status rhqr_pipeline_destroy(rhqr_pipeline p) {
  if (p == nullptr) return RHQR_OK;
  const bool synced = cudaStreamSynchronize(p->s_in) == cudaSuccess &&
                      cudaStreamSynchronize(p->s_comp) == cudaSuccess &&
                      cudaStreamSynchronize(p->s_out) == cudaSuccess;
  release(p);
  return synced ? RHQR_OK : RHQR_ECUDA;
}

}  // extern "C"
