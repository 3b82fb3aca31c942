// Per-tile front-to-back alpha compositing (Eq. 4 with the Gaussian weight of
// Eq. 1).  One 256-thread CTA per 16x16 screen tile, one pixel per thread; warp
// w owns the 8x4 pixel block (w % 2, w / 2) of the tile.  The tile's depth-
// sorted list is walked in batches of 256: each thread gathers one Gaussian into
// shared memory as three 128-bit words -- (x, y, -a/2, -c/2), (-b, exponent
// threshold, opacity, -) and the bounding box of the ellipse where alpha can
// reach 1/255 -- plus its colour.  A warp skips a Gaussian whose box misses its
// block with one uniform branch; pixels inside evaluate Eq. 1 exactly.  The box
// is conservative, so it never changes a decision.  A CTA stops as soon as all
// of its pixels have saturated (__syncthreads_count).
#include "fs4d_internal.cuh"

namespace fs4d {
namespace {

constexpr int kThreads = kTile * kTile;
constexpr int kBatch = kThreads;
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.f / 255.f;
constexpr float kTMin = 1e-4f;

__global__ void __launch_bounds__(kThreads) composite_kernel(int width, int height, int tiles_x,
                                                            const uint2* __restrict__ ranges,
                                                            const uint32_t* __restrict__ values,
                                                            const float2* __restrict__ xy,
                                                            const float4* __restrict__ conic_opacity,
                                                            const float* __restrict__ rgb, float* __restrict__ image,
                                                            float* __restrict__ t_final, int* __restrict__ n_contrib) {
  __shared__ float4 s_g0[kBatch];
  __shared__ float4 s_g1[kBatch];
  __shared__ float4 s_box[kBatch];
  __shared__ float s_rgb[3 * kBatch];
  const int tile = blockIdx.x;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bx0 = tx * kTile + (warp & 1) * 8, by0 = ty * kTile + (warp >> 1) * 4;
  const int px = bx0 + (lane & 7), py = by0 + (lane >> 3);
  const bool inside = px < width && py < height;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  // pixel-centre extent of this warp's block
  const float wx0 = (float)bx0 + 0.5f, wx1 = (float)bx0 + 7.5f, wy0 = (float)by0 + 0.5f, wy1 = (float)by0 + 3.5f;
  const uint2 range = ranges[tile];
  const int n = (int)(range.y - range.x);

  bool done = !inside;
  float T = 1.f, R = 0.f, G = 0.f, B = 0.f;
  int last = 0;
  for (int base = 0; base < n; base += kBatch) {
    if (__syncthreads_count(done) == kThreads) break;
    const int k = base + (int)threadIdx.x;
    if (k < n) {
      const uint32_t g = values[range.x + k];
      const float2 p = xy[g];
      const float4 co = conic_opacity[g];
      const float thr = composite_exp_threshold(co.w);
      s_g0[threadIdx.x] = make_float4(p.x, p.y, -0.5f * co.x, -0.5f * co.z);
      s_g1[threadIdx.x] = make_float4(-co.y, thr, co.w, 0.f);
      // {d : d^T K d <= -2 thr} has half-extents sqrt(-2 thr K^-1_xx), sqrt(-2 thr K^-1_yy)
      float4 box = make_float4(1e30f, -1e30f, 1e30f, -1e30f);  // empty: alpha can never reach 1/255
      const float detk = co.x * co.z - co.y * co.y;
      if (thr < 0.f && !(detk > 0.f)) box = make_float4(-1e30f, 1e30f, -1e30f, 1e30f);  // no bound: test every pixel
      if (thr < 0.f && detk > 0.f) {
        const float s = -2.f * thr;
        const float ex = sqrtf(s * co.z / detk) * 1.001f + 0.01f;
        const float ey = sqrtf(s * co.x / detk) * 1.001f + 0.01f;
        box = make_float4(p.x - ex, p.x + ex, p.y - ey, p.y + ey);
      }
      s_box[threadIdx.x] = box;
      s_rgb[3 * threadIdx.x] = rgb[3 * g];
      s_rgb[3 * threadIdx.x + 1] = rgb[3 * g + 1];
      s_rgb[3 * threadIdx.x + 2] = rgb[3 * g + 2];
    }
    __syncthreads();
    const int m = min(kBatch, n - base);
    for (int j = 0; j < m; ++j) {
      const float4 box = s_box[j];
      if (box.x > wx1 || box.y < wx0 || box.z > wy1 || box.w < wy0) continue;  // warp-uniform
      if (done) continue;
      const float4 g0 = s_g0[j];
      const float4 g1 = s_g1[j];
      const float power = composite_power(g0, g1, g0.x - fx, g0.y - fy);
      if (power > 0.f || power < g1.y) continue;
      const float alpha = fminf(kAlphaMax, g1.z * expf(power));
      if (alpha < kAlphaMin) continue;
      const float Tn = T * (1.f - alpha);
      if (Tn < kTMin) {
        done = true;
        continue;
      }
      const float w = alpha * T;
      R += s_rgb[3 * j] * w;
      G += s_rgb[3 * j + 1] * w;
      B += s_rgb[3 * j + 2] * w;
      T = Tn;
      last = base + j + 1;
    }
  }
  if (inside) {
    const int pix = py * width + px;
    image[3 * pix] = R;
    image[3 * pix + 1] = G;
    image[3 * pix + 2] = B;
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
  composite_kernel<<<tiles_x * tiles_y, kThreads, 0, s>>>(width, height, tiles_x, ranges, values, xy, conic_opacity,
                                                          rgb, image, t_final, n_contrib);
  return cudaGetLastError();
}

}  // namespace fs4d
