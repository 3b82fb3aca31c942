// Per-tile front-to-back alpha compositing (Eq. 4 with the Gaussian weight of
// Eq. 1).  One 256-thread CTA per 16x16 screen tile, one pixel per thread; warp
// w owns the 8x4 pixel block (w % 2, w / 2) of the tile.  The tile's depth-
// sorted list is walked in batches of 256: each thread gathers one Gaussian into
// shared memory as two 128-bit words -- (x, y, -a/2, -c/2) and (-b, exponent
// threshold, opacity, block mask) -- plus its colour, where the mask says which
// of the eight warp blocks the ellipse {alpha >= 1/255} can reach.  A warp skips
// a Gaussian outside its block with one uniform branch; pixels inside evaluate
// Eq. 1 exactly.  The mask is conservative, so it never changes a decision.  A CTA stops as soon as all
// of its pixels have saturated (__syncthreads_count).
#include "fs4d_internal.cuh"

namespace fs4d {
namespace {

constexpr int kThreads = kTile * kTile;
constexpr int kBatch = kThreads;
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.f / 255.f;
constexpr float kTMin = 1e-4f;

// Minimum over t in [t0, t1] of A u^2 + 2 B u t + C t^2 for fixed u (C > 0).
__device__ __forceinline__ float edge_min(float A, float B, float C, float u, float t0, float t1) {
  const float t = fminf(t1, fmaxf(t0, -B * u / C));
  return A * u * u + 2.f * B * u * t + C * t * t;
}

// Bit b set iff some pixel centre of warp block b (8x4 pixels at ((b%2)*8, (b/2)*4)
// of tile (tx, ty)) may reach alpha >= 1/255: the minimum of q(d) = d^T K d over
// the block's pixel-centre rectangle (d relative to the mean) is compared with
// s = -2 * thr.  The minimum of a positive-definite quadratic over a rectangle is
// 0 if the mean lies inside, else on one of the four edges.  A 0.2% + 1e-3
// margin keeps the test conservative against float32 rounding.
__device__ __forceinline__ uint32_t block_mask(float2 p, float4 co, float thr, int tx, int ty) {
  if (!(thr < 0.f)) return 0u;                         // alpha can never reach 1/255
  const float A = co.x, B = co.y, C = co.z;
  if (!(A > 0.f && C > 0.f && A * C - B * B > 0.f)) return 0xffu;  // no usable bound: test every pixel
  const float s = -2.f * thr * 1.002f + 1e-3f;
  uint32_t mask = 0u;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const float x0 = (float)(tx * kTile + (b & 1) * 8) + 0.5f - p.x, x1 = x0 + 7.f;
    const float y0 = (float)(ty * kTile + (b >> 1) * 4) + 0.5f - p.y, y1 = y0 + 3.f;
    float q;
    if (x0 <= 0.f && x1 >= 0.f && y0 <= 0.f && y1 >= 0.f) {
      q = 0.f;
    } else {
      q = fminf(fminf(edge_min(A, B, C, x0, y0, y1), edge_min(A, B, C, x1, y0, y1)),
                fminf(edge_min(C, B, A, y0, x0, x1), edge_min(C, B, A, y1, x0, x1)));
    }
    if (q <= s) mask |= 1u << b;
  }
  return mask;
}

__global__ void __launch_bounds__(kThreads) composite_kernel(int width, int height, int tiles_x,
                                                            const uint2* __restrict__ ranges,
                                                            const uint32_t* __restrict__ values,
                                                            const float2* __restrict__ xy,
                                                            const float4* __restrict__ conic_opacity,
                                                            const float* __restrict__ rgb, float* __restrict__ image,
                                                            float* __restrict__ t_final, int* __restrict__ n_contrib) {
  __shared__ float4 s_g0[kBatch];
  __shared__ float4 s_g1[kBatch];
  __shared__ float s_rgb[3 * kBatch];
  const int tile = blockIdx.x;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bx0 = tx * kTile + (warp & 1) * 8, by0 = ty * kTile + (warp >> 1) * 4;
  const int px = bx0 + (lane & 7), py = by0 + (lane >> 3);
  const bool inside = px < width && py < height;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
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
      s_g1[threadIdx.x] = make_float4(-co.y, thr, co.w, __uint_as_float(block_mask(p, co, thr, tx, ty)));
      s_rgb[3 * threadIdx.x] = rgb[3 * g];
      s_rgb[3 * threadIdx.x + 1] = rgb[3 * g + 1];
      s_rgb[3 * threadIdx.x + 2] = rgb[3 * g + 2];
    }
    __syncthreads();
    const int m = min(kBatch, n - base);
    for (int j = 0; j < m; ++j) {
      const float4 g1 = s_g1[j];
      if (!((__float_as_uint(g1.w) >> warp) & 1u)) continue;  // warp-uniform: ellipse misses the block
      if (done) continue;
      const float4 g0 = s_g0[j];
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
