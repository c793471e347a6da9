// Backward of render_rays: not built yet.
#include "common.cuh"

using namespace tsdfs;

extern "C" size_t tsdfs_backward_workspace_size(const tsdfs_mlp* mlp, int64_t n_rays, int64_t max_samples) {
    (void)mlp;
    (void)n_rays;
    (void)max_samples;
    return 0;
}
extern "C" int render_rays_backward(const tsdfs_mlp*, const float*, const float*, const float*, const float*,
                                    const int32_t*, const uint8_t*, int64_t, int64_t, const float*, const float*, float,
                                    float*, float*, void*, size_t, tsdfs_stream_t) {
    return fail(TSDFS_E_UNSUPPORTED, "backward not built");
}
