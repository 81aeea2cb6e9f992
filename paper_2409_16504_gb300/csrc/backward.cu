// K7/K8: backward of the renderer (filled in below the forward path).
#include "common.cuh"

namespace p2e {
size_t backward_scratch_bytes(int64_t) { return 0; }
cudaError_t launch_render_backward(const p2e_gaussians *, const p2e_projected *, const p2e_bins *,
                                   const Views &, const float *, const uint32_t *, const float *,
                                   const float *, const float *, const float *, float *, float *,
                                   float *, float *, float *, float *, void *, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace p2e
