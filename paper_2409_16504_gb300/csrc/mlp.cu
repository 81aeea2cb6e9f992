// K11: learned per-point estimator (filled in after the closed-form path).
#include "common.cuh"

namespace p2e {
size_t mlp_scratch_bytes(int64_t) { return 256; }
cudaError_t launch_mlp_estimate(const float *, const float *, int64_t, const void *, const uint32_t *,
                                p2e_gaussians *, void *, int, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace p2e
