#include "sketch_tc.cuh"

namespace rhqr {
bool sketch_tc_supported(const SketchView &, int64_t, int32_t) { return false; }
size_t sketch_tc_workspace_bytes(const SketchView &, int64_t, int32_t) { return 0; }
rhqr_status sketch_apply_tc(const SketchView &, int32_t, const float *, int64_t, int64_t, int, double *, int64_t,
                            void *, size_t, cudaStream_t) {
  return RHQR_ENOTSUP;
}
}  // namespace rhqr
