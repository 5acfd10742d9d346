// rhqr_sketch_apply_noalloc: the sketch entry point without a caller
// workspace, for callers that cannot allocate device memory when they call:
// framework hooks and custom operators whose rules forbid device allocation
// at call time, real-time paths that must not block on cudaMalloc, and host
// applications that own all device memory themselves and cannot grant the
// library a workspace.
//
// Its scratch is this file's static device array, which every GPU that loads
// the library holds until the process exits.  Host code cannot pass the
// array's name to a kernel (on the host it only stands for the symbol), so
// the device address is looked up with cudaGetSymbolAddress the first time
// the entry point runs on a device (with that device current) and cached per
// device together with the CUDA context it belongs to; a call in another
// context of that device (after cudaDeviceReset, say) looks it up again.
// That first call should therefore come before any stream capture.  All calls
// share the array and it keeps the previous call's contents: the only field
// that must start at zero (the error flag of the tensor-core kernel) is
// cleared on the stream by every call, and calls whose work overlaps on the
// GPU (different streams, other threads) race on it.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "sketch.cuh"
#include "sketch_tc.cuh"

namespace rhqr {

const SketchView *sketch_view_of(rhqr_sketch s);

static __device__ __align__(256) unsigned char g_noalloc_scratch[RHQR_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[64];
static void *g_noalloc_ctx[64];

// The current CUDA context (driver API, reached through the runtime).
static void *current_context() {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuCtxGetCurrent_v4000)p;
    else
      (void)cudaGetLastError();
    looked = true;
  }
  CUcontext ctx = nullptr;
  if (fn == nullptr || fn(&ctx) != CUDA_SUCCESS) return nullptr;
  return (void *)ctx;
}

// Device address of the scratch array on the current device, looked up once
// per device and context.
static rhqr_status noalloc_scratch(void **out) {
  int dev = 0;
  RHQR_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return RHQR_ENOTSUP;
  void *ctx = current_context();  // NULL before the runtime has set up the device's context
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr || ctx == nullptr || ctx != g_noalloc_ctx[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      (void)cudaGetLastError();
      return RHQR_ECUDA;
    }
    g_noalloc_ptr[dev] = p;
    g_noalloc_ctx[dev] = current_context();  // set up by now
  }
  *out = g_noalloc_ptr[dev];
  return RHQR_OK;
}

}  // namespace rhqr

using namespace rhqr;

extern "C" rhqr_status rhqr_sketch_apply_noalloc(rhqr_sketch s, int32_t m, const void *X, int32_t xt, int64_t n,
                                                 int32_t c, int64_t ldx, double *Z, int64_t ldz,
                                                 rhqr_stream_t stream) {
  if (s == nullptr || X == nullptr || Z == nullptr || c < 1) return RHQR_EINVAL;
  if (xt != RHQR_F64 && xt != RHQR_F32) return RHQR_EINVAL;
  const SketchView &v = *sketch_view_of(s);
  if (m < 0 || n <= m || m > v.k) return RHQR_EINVAL;
  if (v.kind == RHQR_SKETCH_GAUSSIAN && n != v.n) return RHQR_EINVAL;
  if (v.kind == RHQR_SKETCH_SRHT && n > v.N) return RHQR_EINVAL;
  if (ldx < n || ldz < (int64_t)v.k + m) return RHQR_EINVAL;
  const bool tc = xt == RHQR_F32 && sketch_tc_supported(v, n, m, c) && ldx % 4 == 0 && ((uintptr_t)X % 16) == 0;
  const size_t need = tc ? sketch_tc_workspace_bytes(v, n, m, c) : sketch_apply_workspace_bytes(v, m, xt, n, c);
  if (need > (size_t)RHQR_NOALLOC_SCRATCH_BYTES) return RHQR_ENOMEM;  // beyond the fixed scratch
  void *ws = nullptr;
  RHQR_TRY(noalloc_scratch(&ws));
  cudaStream_t st = (cudaStream_t)stream;
  if (tc)
    return sketch_apply_tc(v, m, (const float *)X, n, c, ldx, 3, Z, ldz, ws, RHQR_NOALLOC_SCRATCH_BYTES, nullptr, 0, st);
  return sketch_apply_simt(v, m, X, xt, n, c, ldx, Z, ldz, ws, RHQR_NOALLOC_SCRATCH_BYTES, st);
}
