// Per-tile front-to-back alpha compositing (Eq. 4 with the Gaussian weight of
// Eq. 1).  One 256-thread CTA per 16x16 screen tile, one pixel per thread.  The
// tile's depth-sorted list is walked in batches of 256 Gaussians: each thread
// gathers one Gaussian's (xy, conic, opacity, rgb) into shared memory, then
// every pixel blends the batch from shared memory.  A CTA stops as soon as all
// of its pixels have saturated (__syncthreads_count), so a batch is only
// gathered while some pixel still needs it.
#include "fs4d_internal.cuh"

namespace fs4d {
namespace {

constexpr int kBatch = kTile * kTile;
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.f / 255.f;
constexpr float kTMin = 1e-4f;

__global__ void __launch_bounds__(kBatch) composite_kernel(int width, int height, int tiles_x,
                                                          const uint2* __restrict__ ranges,
                                                          const uint32_t* __restrict__ values,
                                                          const float2* __restrict__ xy,
                                                          const float4* __restrict__ conic_opacity,
                                                          const float* __restrict__ rgb, float* __restrict__ image,
                                                          float* __restrict__ t_final, int* __restrict__ n_contrib) {
  __shared__ float2 s_xy[kBatch];
  __shared__ float4 s_co[kBatch];
  __shared__ float s_rgb[3 * kBatch];
  const int tile = blockIdx.x;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int px = tx * kTile + (threadIdx.x % kTile), py = ty * kTile + (threadIdx.x / kTile);
  const bool inside = px < width && py < height;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  const uint2 range = ranges[tile];
  const int n = (int)(range.y - range.x);

  bool done = !inside;
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
  int last = 0;
  for (int base = 0; base < n; base += kBatch) {
    if (__syncthreads_count(done) == kBatch) break;
    const int k = base + (int)threadIdx.x;
    if (k < n) {
      const uint32_t g = values[range.x + k];
      s_xy[threadIdx.x] = xy[g];
      s_co[threadIdx.x] = conic_opacity[g];
      s_rgb[3 * threadIdx.x] = rgb[3 * g];
      s_rgb[3 * threadIdx.x + 1] = rgb[3 * g + 1];
      s_rgb[3 * threadIdx.x + 2] = rgb[3 * g + 2];
    }
    __syncthreads();
    const int m = min(kBatch, n - base);
    for (int j = 0; !done && j < m; ++j) {
      const float2 p = s_xy[j];
      const float4 co = s_co[j];
      const float dx = p.x - fx, dy = p.y - fy;
      const float power = -0.5f * (co.x * dx * dx + co.z * dy * dy) - co.y * dx * dy;
      if (power > 0.f) continue;
      const float alpha = fminf(kAlphaMax, co.w * expf(power));
      if (alpha < kAlphaMin) continue;
      const float Tn = T * (1.f - alpha);
      if (Tn < kTMin) {
        done = true;
        break;
      }
      const float wgt = alpha * T;
      C0 += s_rgb[3 * j] * wgt;
      C1 += s_rgb[3 * j + 1] * wgt;
      C2 += s_rgb[3 * j + 2] * wgt;
      T = Tn;
      last = base + j + 1;
    }
  }
  if (inside) {
    const int pix = py * width + px;
    image[3 * pix] = C0;
    image[3 * pix + 1] = C1;
    image[3 * pix + 2] = C2;
    if (t_final) t_final[pix] = T;
    if (n_contrib) n_contrib[pix] = last;
  }
}

}  // namespace

cudaError_t launch_composite(int width, int height, const uint2* ranges, const uint32_t* values, const float2* xy,
                             const float4* conic_opacity, const float* rgb, float* image, float* t_final,
                             int* n_contrib, cudaStream_t s) {
  const int tiles_x = (width + kTile - 1) / kTile, tiles_y = (height + kTile - 1) / kTile;
  if (tiles_x * tiles_y == 0) return cudaSuccess;
  composite_kernel<<<tiles_x * tiles_y, kBatch, 0, s>>>(width, height, tiles_x, ranges, values, xy, conic_opacity,
                                                        rgb, image, t_final, n_contrib);
  return cudaGetLastError();
}

}  // namespace fs4d
