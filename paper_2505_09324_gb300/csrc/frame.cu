// Frame input: 8-bit interleaved RGB (the layout video decoders and cameras
// deliver) to the planar float frame the fit loop reads, on the device, so a
// frame crosses the host link as 3 bytes per pixel instead of 12.
#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

// One thread per pixel: three byte loads (consecutive threads read
// consecutive bytes), three coalesced plane stores.
__global__ void __launch_bounds__(256)
k_frame_from_rgb8(const uint8_t* __restrict__ rgb, int width, int height, int64_t row_bytes,
                  float* __restrict__ frame) {
  pdl_begin();
  const int64_t hw = (int64_t)width * height;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < hw;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = i / width, x = i - y * width;
    const uint8_t* px = rgb + y * row_bytes + 3 * x;
    frame[i] = __fdiv_rn((float)px[0], 255.0f);
    frame[hw + i] = __fdiv_rn((float)px[1], 255.0f);
    frame[2 * hw + i] = __fdiv_rn((float)px[2], 255.0f);
  }
}

}  // namespace
}  // namespace gs2d

using namespace gs2d;

extern "C" gs2d_status gs2d_frame_from_rgb8(const uint8_t* rgb, int32_t width, int32_t height,
                                            int64_t row_bytes, float* frame, void* stream) {
  if (width < 0 || height < 0 || (width > 0 && height > 0 && (!rgb || !frame)) ||
      row_bytes < 3 * (int64_t)width)
    return set_error(GS2D_ERR_INVALID_ARG, "gs2d_frame_from_rgb8: arguments");
  const int64_t hw = (int64_t)width * height;
  if (hw == 0) return set_error(GS2D_OK, "");
  const int64_t want = (hw + 255) / 256;
  const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
  const cudaError_t e = launch_pdl(k_frame_from_rgb8, blocks, 256, 0, (cudaStream_t)stream, rgb,
                                   (int)width, (int)height, row_bytes, frame);
  if (e != cudaSuccess) return set_error(GS2D_ERR_CUDA, cudaGetErrorString(e));
  return set_error(GS2D_OK, "");
}
