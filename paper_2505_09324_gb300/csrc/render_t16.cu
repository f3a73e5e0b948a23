// Render kernels for 16x16 tiles (all stages and modes; see render_impl.cuh).
#include "render_impl.cuh"

namespace gs2d {

cudaError_t launch_render_t16(int stage, int launch, RenderMode mode, const RenderArgs& a,
                              cudaStream_t s) {
  return launch_tile<16>(stage, launch, mode, a, s);
}

cudaError_t prime_render_t16(int stage, int launch) { return prime_tile<16>(stage, launch); }

}  // namespace gs2d
