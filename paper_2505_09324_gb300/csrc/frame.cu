// Frame input: 8-bit interleaved RGB (the layout video decoders and cameras
// deliver) to the planar float frame the fit loop reads, on the device, so a
// frame crosses the host link as 3 bytes per pixel instead of 12.
#include "gs2d_internal.cuh"

namespace gs2d {
namespace {

// One thread per four consecutive pixels of a row (blockIdx.y = row): twelve
// bytes in (three aligned words where the row allows), three 16-byte plane
// stores where the width allows; the same division per value either way.
// No integer division per pixel: the row comes from the grid.
__global__ void __launch_bounds__(256)
k_frame_from_rgb8(const uint8_t* __restrict__ rgb, int width, int height, int64_t row_bytes,
                  float* __restrict__ frame) {
  pdl_begin();
  const int y = blockIdx.y;
  const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (x0 >= width) return;
  const int64_t hw = (int64_t)width * height, o = (int64_t)y * width + x0;
  const uint8_t* px = rgb + (int64_t)y * row_bytes + 3 * (int64_t)x0;
  const bool vec = (width & 3) == 0 && (row_bytes & 3) == 0 && x0 + 4 <= width &&
                   (reinterpret_cast<uintptr_t>(rgb) & 3) == 0 &&
                   (reinterpret_cast<uintptr_t>(frame) & 15) == 0;
  if (vec) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(px);
    const uint32_t b[3] = {w[0], w[1], w[2]};
    float c[12];
#pragma unroll
    for (int k = 0; k < 12; k++)
      c[k] = __fdiv_rn((float)((b[k >> 2] >> (8 * (k & 3))) & 0xFFu), 255.0f);
#pragma unroll
    for (int p = 0; p < 3; p++)
      *reinterpret_cast<float4*>(frame + p * hw + o) =
          make_float4(c[p], c[3 + p], c[6 + p], c[9 + p]);
    return;
  }
  for (int k = 0; k < 4 && x0 + k < width; k++) {
    frame[o + k] = __fdiv_rn((float)px[3 * k], 255.0f);
    frame[hw + o + k] = __fdiv_rn((float)px[3 * k + 1], 255.0f);
    frame[2 * hw + o + k] = __fdiv_rn((float)px[3 * k + 2], 255.0f);
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
  if (height > 65535) return set_error(GS2D_ERR_INVALID_ARG, "gs2d_frame_from_rgb8: height");
  const dim3 grid((unsigned)((width + 1023) / 1024), (unsigned)height);
  const cudaError_t e = launch_pdl(k_frame_from_rgb8, grid, 256, 0, (cudaStream_t)stream, rgb,
                                   (int)width, (int)height, row_bytes, frame);
  if (e != cudaSuccess) return set_error(GS2D_ERR_CUDA, cudaGetErrorString(e));
  return set_error(GS2D_OK, "");
}
