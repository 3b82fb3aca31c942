// Per-tile front-to-back alpha compositing (Eq. 4 with the Gaussian weight of
// Eq. 1).  One 256-thread CTA per 16x16 screen tile (optionally in a given launch
// order, longest lists first), one pixel per thread; warp
// w owns the 8x4 pixel block (w % 2, w / 2) of the tile.  The tile's depth-
// sorted list is walked in batches of 256: each thread gathers one Gaussian into
// shared memory -- position and log2-scaled conic, opacity and colour -- and the
// 8-bit mask of the warp blocks that the ellipse {alpha >= 1/255} can reach.
// Each warp then compacts the batch to the Gaussians whose mask holds its block
// (ballot + popc, order kept) and walks only those; every pixel evaluates Eq. 1
// exactly for them.  The mask is conservative, so it never changes a decision.
// A warp whose pixels have all saturated skips the batch; a CTA stops as soon as
// all of its pixels have (__syncthreads_count).  Batches alternate between two
// staging buffers, so one barrier per batch suffices.
#include "fs4d_internal.cuh"

namespace fs4d {
namespace {

constexpr int kThreads = kTile * kTile;
constexpr int kBatch = kThreads;
constexpr int kWarps = kThreads / 32;
constexpr float kTMin = 1e-4f;
constexpr int kMinBlocks = 5;  // CTAs per SM the register budget must allow

// Bit b set iff some pixel centre of warp block b (8x4 pixels at ((b%2)*8, (b/2)*4)
// of tile (tx, ty)) may reach alpha >= 1/255: the minimum of q(d) = d^T K d over
// the block's pixel-centre rectangle (d relative to the mean) is compared with
// s = -2 * thr.  The minimum of a positive-definite quadratic over a rectangle is
// 0 if the mean lies inside, else on one of the four edges (each minimised in
// closed form, rect_min).  If
// all four corner pixel centres of the tile lie in the ellipse q <= s, so does the
// whole tile (the ellipse is convex) and every block is set at once.  A 0.2% +
// 1e-3 margin keeps the test conservative against float32 rounding.
__device__ __forceinline__ uint32_t block_mask(float2 p, float4 co, float thr, int tx, int ty) {
  if (!(thr < 0.f)) return 0u;                         // alpha can never reach 1/255
  const float A = co.x, B = co.y, C = co.z;
  if (!(A > 0.f && C > 0.f && A * C - B * B > 0.f)) return 0xffu;  // no usable bound: test every pixel
  const float s = -2.f * thr * 1.002f + 1e-3f;
  const float X0 = (float)(tx * kTile) + 0.5f - p.x, X1 = X0 + (float)(kTile - 1);
  const float Y0 = (float)(ty * kTile) + 0.5f - p.y, Y1 = Y0 + (float)(kTile - 1);
  auto q = [&](float x, float y) { return A * x * x + 2.f * B * x * y + C * y * y; };
  if (fmaxf(fmaxf(q(X0, Y0), q(X1, Y0)), fmaxf(q(X0, Y1), q(X1, Y1))) <= s) return 0xffu;
  const float kx = -B / C, ky = -B / A;
  uint32_t mask = 0u;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const float x0 = X0 + (float)((b & 1) * 8), x1 = x0 + 7.f;
    const float y0 = Y0 + (float)((b >> 1) * 4), y1 = y0 + 3.f;
    if (rect_min(A, B, C, kx, ky, x0, x1, y0, y1) <= s) mask |= 1u << b;
  }
  return mask;
}

// One staged batch of m Gaussians (list positions base .. base + m - 1) for the
// calling thread's pixel: the warp compacts the batch to the Gaussians whose mask
// holds its block (ballot, order kept) and walks them two per step -- both weights
// are evaluated before the two (sequential, front-to-back) transmittance updates.
// AUX: track each pixel's last contributor.
template <bool AUX>
__device__ __forceinline__ void composite_batch(int m, int base, const float4* s_g0, const float4* s_g1,
                                                const float* s_blue, const uint32_t* s_mask, uint8_t* list,
                                                int warp, int lane, float fx, float fy, bool& done, float& T,
                                                float& R, float& G, float& B, int& last) {
  const uint32_t lane_lt = (1u << lane) - 1u;
  int cnt = 0;
  for (int c0 = 0; c0 < m; c0 += 32) {
    const int j = c0 + lane;
    const bool hit = j < m && ((s_mask[j] >> warp) & 1u);
    const uint32_t bal = __ballot_sync(0xffffffffu, hit);
    if (hit) list[cnt + __popc(bal & lane_lt)] = (uint8_t)j;
    cnt += __popc(bal);
  }
  __syncwarp();
  for (int i = 0; i < cnt && !done; i += 2) {
    const int ja = list[i];
    const bool has_b = i + 1 < cnt;
    const int jb = has_b ? list[i + 1] : ja;
    const float4 a0 = s_g0[ja], a1 = s_g1[ja];
    const float4 b0 = s_g0[jb], b1 = s_g1[jb];
    float ga, gb;
    const float alpha_a = composite_alpha(a0, a1.x, a1.y, a0.x - fx, a0.y - fy, ga);
    float alpha_b = composite_alpha(b0, b1.x, b1.y, b0.x - fx, b0.y - fy, gb);
    if (!has_b) alpha_b = 0.f;
    if (alpha_a > 0.f) {
      const float Tn = T * (1.f - alpha_a);
      if (Tn < kTMin) {
        done = true;
        break;
      }
      const float w = alpha_a * T;
      R += a1.z * w;
      G += a1.w * w;
      B += s_blue[ja] * w;
      T = Tn;
      if (AUX) last = base + ja + 1;
    }
    if (alpha_b > 0.f) {
      const float Tn = T * (1.f - alpha_b);
      if (Tn < kTMin) {
        done = true;
        break;
      }
      const float w = alpha_b * T;
      R += b1.z * w;
      G += b1.w * w;
      B += s_blue[jb] * w;
      T = Tn;
      if (AUX) last = base + jb + 1;
    }
  }
  __syncwarp();
}

// Stage Gaussian g of a batch into slot k.
__device__ __forceinline__ void stage_gaussian(int k, uint32_t g, const float2* __restrict__ xy,
                                               const float4* __restrict__ conic_opacity,
                                               const float* __restrict__ rgb, int tx, int ty, float4* s_g0,
                                               float4* s_g1, float* s_blue, uint32_t* s_mask) {
  const float2 p = xy[g];
  const float4 co = conic_opacity[g];
  s_g0[k] = composite_coeffs(p, co);
  s_g1[k] = make_float4(composite_b2(co), co.w, rgb[3 * g], rgb[3 * g + 1]);
  s_blue[k] = rgb[3 * g + 2];
  s_mask[k] = block_mask(p, co, composite_exp_threshold(co.w), tx, ty);
}

__device__ __forceinline__ void write_pixel(bool inside, int px, int py, int width, float R, float G, float B,
                                            float T, int last, float* image, float* t_final, int* n_contrib,
                                            bool aux) {
  if (!inside) return;
  const int pix = py * width + px;
  image[3 * pix] = R;
  image[3 * pix + 1] = G;
  image[3 * pix + 2] = B;
  if (aux) {
    if (t_final) t_final[pix] = T;
    if (n_contrib) n_contrib[pix] = last;
  }
}

// Tile lists as [start, end) ranges into a list of Gaussian indices.
template <bool AUX>
__global__ void __launch_bounds__(kThreads, kMinBlocks) composite_kernel(int width, int height, int tiles_x,
                                                            const uint2* __restrict__ ranges,
                                                            const uint32_t* __restrict__ values,
                                                            const float2* __restrict__ xy,
                                                            const float4* __restrict__ conic_opacity,
                                                            const float* __restrict__ rgb, float* __restrict__ image,
                                                            float* __restrict__ t_final, int* __restrict__ n_contrib,
                                                            const uint32_t* __restrict__ order, int vstride) {
  // two staging buffers: batch i is staged while batch i - 1 may still be read
  __shared__ float4 s_g0b[2][kBatch];   // x, y, a2, c2
  __shared__ float4 s_g1b[2][kBatch];   // b2, opacity, red, green
  __shared__ float s_blueb[2][kBatch];
  __shared__ uint32_t s_maskb[2][kBatch];
  __shared__ uint8_t s_list[kWarps][kBatch];
  pdl_wait();
  pdl_trigger();
  const int tile = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
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
  for (int base = 0, it = 0; base < n; base += kBatch, ++it) {
    const int b = it & 1;
    const int k = base + (int)threadIdx.x;
    if (k < n)
      stage_gaussian(threadIdx.x, values[(size_t)vstride * (range.x + k)], xy, conic_opacity, rgb, tx, ty, s_g0b[b], s_g1b[b],
                     s_blueb[b], s_maskb[b]);
    // one barrier per batch: this batch is staged, the buffer staged next was
    // last read for batch i - 1, which every thread has finished; and if every
    // pixel has saturated the tile is done
    if (__syncthreads_count(done) == kThreads) break;
    if (__all_sync(0xffffffffu, done)) continue;  // warp-uniform
    composite_batch<AUX>(min(kBatch, n - base), base, s_g0b[b], s_g1b[b], s_blueb[b], s_maskb[b], s_list[warp],
                         warp, lane, fx, fy, done, T, R, G, B, last);
  }
  write_pixel(inside, px, py, width, R, G, B, T, last, image, t_final, n_contrib, AUX);
}

}  // namespace

cudaError_t launch_composite(int width, int height, const uint2* ranges, const uint32_t* values, const float2* xy,
                             const float4* conic_opacity, const float* rgb, float* image, float* t_final,
                             int* n_contrib, cudaStream_t s, const uint32_t* order, int values_stride) {
  const int tiles_x = (width + kTile - 1) / kTile, tiles_y = (height + kTile - 1) / kTile;
  if (tiles_x * tiles_y == 0) return cudaSuccess;
  if (t_final || n_contrib)
    return launch_pdl(composite_kernel<true>, tiles_x * tiles_y, kThreads, 0, s, width, height, tiles_x, ranges, values,
                      xy, conic_opacity, rgb, image, t_final, n_contrib, order, values_stride);
  return launch_pdl(composite_kernel<false>, tiles_x * tiles_y, kThreads, 0, s, width, height, tiles_x, ranges, values,
                    xy, conic_opacity, rgb, image, t_final, n_contrib, order, values_stride);
}

}  // namespace fs4d
