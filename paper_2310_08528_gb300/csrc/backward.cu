// Backward of the render path (training, Sec. 4.3): the chain rule of
// compositing (Eq. 4 with Eq. 1), EWA projection (Eq. 2, Eq. 3) with SH colour,
// the deformation update (Eq. 6), the MLP heads and phi_d, and the HexPlane
// sampling (Eq. 5).  Float32 throughout.
//
//  composite_bwd_kernel  one CTA per tile, one pixel per thread, walking the
//      tile's list back to front from each pixel's last blended term.  The
//      contributions of the 256 pixels to each Gaussian are summed inside the
//      CTA (warp shuffles, then shared-memory adds) and written ONCE per
//      (tile, Gaussian) pair into that pair's emission slot, so no global
//      atomics are needed: a Gaussian's slots are contiguous (offsets[g] ...
//      offsets[g] + rect area).
//  project_bwd_kernel    one thread per Gaussian: sums its pair slots, then
//      back-propagates through the conic inverse, Sigma' = A A^T + 0.3 I with
//      A = J W R S, the quaternion normalisation, the perspective Jacobian, the
//      projected mean and the SH colour.
//  mlp_bwd_kernel        one thread per Gaussian: recomputes the deformation
//      forward, back-propagates through the heads and phi_d, stores the layer
//      inputs and deltas feature-major for the weight gradients, and scatters
//      the feature gradient into the plane cells (128-bit float atomics: many
//      Gaussians share a cell).
//  wgrad kernels         dW = D X^T over all Gaussians as per-chunk partial sums
//      followed by a fixed-order reduction (deterministic).
#include <algorithm>

#include "fs4d_internal.cuh"

namespace fs4d {
namespace {

constexpr int kBatch = kTile * kTile;
constexpr float kAlphaMax = 0.99f;
constexpr float kGuard = 1.3f;

// ------------------------------------------------------------------ compositing

// Bit w set iff some pixel centre of the 16x2 pixel rows (2w, 2w + 1) of tile
// (tx, ty) -- warp w's pixels -- may reach alpha >= 1/255 (the rectangle minimum of
// d^T K d against -2 thr with a 0.2% + 1e-3 margin, as the forward's block masks):
// a warp skips, as a whole, the terms whose bit is clear, which no lane of it blends.
__device__ __forceinline__ uint32_t row_pair_mask(float2 p, float4 co, int tx, int ty) {
  const float thr = composite_exp_threshold(co.w);
  if (!(thr < 0.f)) return 0u;
  const float A = co.x, B = co.y, C = co.z;
  if (!(A > 0.f && C > 0.f && A * C - B * B > 0.f)) return 0xffu;
  const float s = -2.f * thr * 1.002f + 1e-3f;
  const float kx = -B / C, ky = -B / A;
  const float X0 = (float)(tx * kTile) + 0.5f - p.x, X1 = X0 + (float)(kTile - 1);
  const float Y0 = (float)(ty * kTile) + 0.5f - p.y;
  uint32_t mask = 0u;
#pragma unroll
  for (int w = 0; w < kBatch / 32; ++w) {
    const float y0 = Y0 + 2.f * (float)w;
    if (rect_min(A, B, C, kx, ky, X0, X1, y0, y0 + 1.f) <= s) mask |= 1u << w;
  }
  return mask;
}

// The warp's sums of nine per-lane values with 14 shuffles instead of 45: values
// 0..7 are halved at each of the offsets 16, 8, 4 (a lane keeps one half and sends
// the other to its partner) and the last one summed over offsets 2 and 1, so lane
// 4k returns the sum of value k (k < 8); the sum of value 8 comes back in s8.
__device__ __forceinline__ float warp_sum9(const float (&v)[kPairGrad], unsigned lane, float& s8) {
  static_assert(kPairGrad == 9, "eight halved values and one summed whole");
  float h4[4], h2[2];
  const bool u16 = (lane & 16u) != 0u, u8 = (lane & 8u) != 0u, u4 = (lane & 4u) != 0u;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    h4[i] = (u16 ? v[i + 4] : v[i]) + __shfl_xor_sync(0xffffffffu, u16 ? v[i] : v[i + 4], 16);
#pragma unroll
  for (int i = 0; i < 2; ++i)
    h2[i] = (u8 ? h4[i + 2] : h4[i]) + __shfl_xor_sync(0xffffffffu, u8 ? h4[i] : h4[i + 2], 8);
  float h1 = (u4 ? h2[1] : h2[0]) + __shfl_xor_sync(0xffffffffu, u4 ? h2[0] : h2[1], 4);
  h1 += __shfl_xor_sync(0xffffffffu, h1, 2);
  h1 += __shfl_xor_sync(0xffffffffu, h1, 1);
  float w = v[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  s8 = w;
  return h1;
}

__global__ void __launch_bounds__(kBatch) composite_bwd_kernel(CompositeBwdArgs a) {
  __shared__ float2 s_xy[kBatch];
  __shared__ float4 s_co[kBatch];
  __shared__ float s_rgb[3 * kBatch];
  __shared__ uint32_t s_slot[kBatch];
  __shared__ uint32_t s_mask[kBatch];
  __shared__ float s_acc[kBatch][kPairGrad];
  __shared__ int s_max_last;
  const int tile = blockIdx.x;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int px = tx * kTile + (threadIdx.x % kTile), py = ty * kTile + (threadIdx.x / kTile);
  const bool inside = px < a.width && py < a.height;
  const int pix = py * a.width + px;
  const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
  const uint2 range = a.ranges[tile];
  const int n = (int)(range.y - range.x);
  const int last = inside ? a.n_contrib[pix] : 0;
  float T = inside ? a.t_final[pix] : 1.f;
  float dC0 = 0.f, dC1 = 0.f, dC2 = 0.f;
  if (inside) {
    dC0 = a.dl_dimage[3 * pix];
    dC1 = a.dl_dimage[3 * pix + 1];
    dC2 = a.dl_dimage[3 * pix + 2];
  }
  float b0 = 0.f, b1 = 0.f, b2 = 0.f;  // colour blended behind the current term
  if (threadIdx.x == 0) s_max_last = 0;
  __syncthreads();
  atomicMax(&s_max_last, last);
  __syncthreads();
  const int max_last = min(s_max_last, n);
  const unsigned lane = threadIdx.x & 31u;

  for (int bstart = ((max_last - 1) / kBatch) * kBatch; bstart >= 0 && max_last > 0; bstart -= kBatch) {
    __syncthreads();
    const int j = bstart + (int)threadIdx.x;
    if (j < n) {
      const uint32_t g = a.values[range.x + j];
      s_xy[threadIdx.x] = a.xy[g];
      const float4 cog = a.conic_opacity[g];
      s_co[threadIdx.x] = cog;
      s_rgb[3 * threadIdx.x] = a.rgb[3 * g];
      s_rgb[3 * threadIdx.x + 1] = a.rgb[3 * g + 1];
      s_rgb[3 * threadIdx.x + 2] = a.rgb[3 * g + 2];
      const int4 r = a.rect[g];
      s_slot[threadIdx.x] = a.offsets[g] + (uint32_t)((ty - r.y) * (r.z - r.x) + (tx - r.x));
      s_mask[threadIdx.x] = row_pair_mask(s_xy[threadIdx.x], cog, tx, ty);
    }
#pragma unroll
    for (int k = 0; k < kPairGrad; ++k) s_acc[threadIdx.x][k] = 0.f;
    __syncthreads();
    const int jend = min(kBatch, max_last - bstart);
    const unsigned warp_bit = 1u << (threadIdx.x >> 5);
    for (int jj = jend - 1; jj >= 0; --jj) {
      if (!(s_mask[jj] & warp_bit)) continue;  // warp-uniform: no pixel of this warp blends term jj
      float gr[kPairGrad];
#pragma unroll
      for (int k = 0; k < kPairGrad; ++k) gr[k] = 0.f;
      bool contrib = false;
      if (bstart + jj < last) {
        const float2 p = s_xy[jj];
        const float4 co = s_co[jj];
        const float4 g0 = composite_coeffs(p, co);
        const float dx = g0.x - fx, dy = g0.y - fy;
        float G;
        const float alpha = composite_alpha(g0, composite_b2(co), co.w, dx, dy, G);
        if (alpha > 0.f) {
          const float a_raw = co.w * G;
          contrib = true;
          const float inv = 1.f / (1.f - alpha);
          const float Ti = T * inv;
          const float c0 = s_rgb[3 * jj], c1 = s_rgb[3 * jj + 1], c2 = s_rgb[3 * jj + 2];
          const float dalpha =
              dC0 * (c0 * Ti - b0 * inv) + dC1 * (c1 * Ti - b1 * inv) + dC2 * (c2 * Ti - b2 * inv);
          const float w = alpha * Ti;
          gr[6] = dC0 * w;
          gr[7] = dC1 * w;
          gr[8] = dC2 * w;
          b0 += c0 * w;
          b1 += c1 * w;
          b2 += c2 * w;
          T = Ti;
          if (a_raw <= kAlphaMax) {
            const float dpow = dalpha * co.w * G;
            gr[0] = -dpow * (co.x * dx + co.y * dy);
            gr[1] = -dpow * (co.z * dy + co.y * dx);
            gr[2] = -0.5f * dpow * dx * dx;
            gr[3] = -dpow * dx * dy;
            gr[4] = -0.5f * dpow * dy * dy;
            gr[5] = dalpha * G;
          }
        }
      }
      const unsigned mask = __ballot_sync(0xffffffffu, contrib);
      if (mask == 0u) continue;
      if (__popc(mask) > 4) {
        float s8;
        const float sk = warp_sum9(gr, lane, s8);
        if ((lane & 3u) == 0u) atomicAdd(&s_acc[jj][lane >> 2], sk);
        if (lane == 0u) atomicAdd(&s_acc[jj][8], s8);
      } else if (contrib) {
#pragma unroll
        for (int k = 0; k < kPairGrad; ++k) atomicAdd(&s_acc[jj][k], gr[k]);
      }
    }
    __syncthreads();
    if ((int)threadIdx.x < jend && bstart + (int)threadIdx.x < n) {
      float4* dst = reinterpret_cast<float4*>(a.grad_pair + (size_t)s_slot[threadIdx.x] * kPairStride);
      const float* v = s_acc[threadIdx.x];
      dst[0] = make_float4(v[0], v[1], v[2], v[3]);
      dst[1] = make_float4(v[4], v[5], v[6], v[7]);
      dst[2] = make_float4(v[8], 0.f, 0.f, 0.f);
    }
  }
}

// ------------------------------------------------------------------ projection

// Real SH basis and its derivative with respect to the direction components,
// differentiating the same formulas the forward evaluates.
constexpr float kY00 = 0.28209479177387814f, kY1 = 0.48860251190291992f, kY2a = 1.0925484305920792f,
                kY20 = 0.31539156525252005f, kY22 = 0.54627421529603959f, kY33 = 0.59004358992664352f,
                kY32 = 2.8906114426405538f, kY31 = 0.45704579946446572f, kY30 = 0.37317633259011540f,
                kY32b = 1.4453057213202769f;

__device__ void sh_basis_and_grad(int deg, float x, float y, float z, float* Y, float (*dY)[3]) {
#pragma unroll
  for (int k = 0; k < 16; ++k) Y[k] = dY[k][0] = dY[k][1] = dY[k][2] = 0.f;
  Y[0] = kY00;
  if (deg < 1) return;
  Y[1] = kY1 * y; Y[2] = kY1 * z; Y[3] = kY1 * x;
  dY[1][1] = kY1; dY[2][2] = kY1; dY[3][0] = kY1;
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kY2a * x * y; dY[4][0] = kY2a * y; dY[4][1] = kY2a * x;
  Y[5] = kY2a * y * z; dY[5][1] = kY2a * z; dY[5][2] = kY2a * y;
  Y[6] = kY20 * (3.f * zz - 1.f); dY[6][2] = 6.f * kY20 * z;
  Y[7] = kY2a * x * z; dY[7][0] = kY2a * z; dY[7][2] = kY2a * x;
  Y[8] = kY22 * (xx - yy); dY[8][0] = 2.f * kY22 * x; dY[8][1] = -2.f * kY22 * y;
  if (deg < 3) return;
  Y[9] = kY33 * y * (3.f * xx - yy); dY[9][0] = 6.f * kY33 * x * y; dY[9][1] = kY33 * (3.f * xx - 3.f * yy);
  Y[10] = kY32 * x * y * z; dY[10][0] = kY32 * y * z; dY[10][1] = kY32 * x * z; dY[10][2] = kY32 * x * y;
  Y[11] = kY31 * y * (5.f * zz - 1.f); dY[11][1] = kY31 * (5.f * zz - 1.f); dY[11][2] = 10.f * kY31 * y * z;
  Y[12] = kY30 * z * (5.f * zz - 3.f); dY[12][2] = kY30 * (15.f * zz - 3.f);
  Y[13] = kY31 * x * (5.f * zz - 1.f); dY[13][0] = kY31 * (5.f * zz - 1.f); dY[13][2] = 10.f * kY31 * x * z;
  Y[14] = kY32b * z * (xx - yy); dY[14][0] = 2.f * kY32b * x * z; dY[14][1] = -2.f * kY32b * y * z;
  dY[14][2] = kY32b * (xx - yy);
  Y[15] = kY33 * x * (xx - 3.f * yy); dY[15][0] = kY33 * (3.f * xx - 3.f * yy); dY[15][1] = -6.f * kY33 * x * y;
}

// The SH colour's backward for one Gaussian with K coefficients per channel: the
// row of 3K coefficients read once (128-bit loads where the rows are 16-byte
// aligned: K = 4, 16), dL/dSH accumulated into g_sh with the same access width,
// and the gradient with respect to the view direction.
template <int K>
__device__ __forceinline__ void sh_colour_bwd(const ProjectBwdArgs& a, int g, const float (&Y)[16],
                                              const float (&dY)[16][3], const float (&G9)[kPairGrad],
                                              float& gdir0, float& gdir1, float& gdir2) {
  constexpr int F = 3 * K;
  constexpr bool kVec = (F % 4) == 0;
  float shv[F];
  const float* row = a.sh + (size_t)g * F;
  if (kVec) {
#pragma unroll
    for (int i = 0; i < F / 4; ++i) {
      const float4 v = reinterpret_cast<const float4*>(row)[i];
      shv[4 * i] = v.x; shv[4 * i + 1] = v.y; shv[4 * i + 2] = v.z; shv[4 * i + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < F; ++i) shv[i] = row[i];
  }
  float gsh[F];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float raw = 0.5f;
#pragma unroll
    for (int k = 0; k < K; ++k) raw += Y[k] * shv[3 * k + ch];
    const bool live = raw > 0.f;  // clamped at 0: no gradient
    const float gr = live ? G9[6 + ch] : 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      gsh[3 * k + ch] = gr * Y[k];
      const float s = gr * shv[3 * k + ch];
      gdir0 += s * dY[k][0];
      gdir1 += s * dY[k][1];
      gdir2 += s * dY[k][2];
    }
  }
  if (!a.g_sh) return;
  float* out = a.g_sh + (size_t)g * F;
  if (kVec) {
#pragma unroll
    for (int i = 0; i < F / 4; ++i) {
      float4 v = reinterpret_cast<float4*>(out)[i];
      v.x += gsh[4 * i]; v.y += gsh[4 * i + 1]; v.z += gsh[4 * i + 2]; v.w += gsh[4 * i + 3];
      reinterpret_cast<float4*>(out)[i] = v;
    }
  } else {
#pragma unroll
    for (int i = 0; i < F; ++i) out[i] += gsh[i];
  }
}

__global__ void __launch_bounds__(128) project_bwd_kernel(ProjectBwdArgs a) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.n) return;
  float* gd = a.gd + 10 * (size_t)g;
  if (a.radius[g] == 0) {
#pragma unroll
    for (int k = 0; k < 10; ++k) gd[k] = 0.f;
    return;
  }
  // sum the pair slots of this Gaussian (contiguous by construction)
  const int4 rc = a.rect[g];
  const uint32_t e0 = a.offsets[g], cnt = (uint32_t)((rc.z - rc.x) * (rc.w - rc.y));
  float G9[kPairGrad];
#pragma unroll
  for (int k = 0; k < kPairGrad; ++k) G9[k] = 0.f;
  for (uint32_t e = 0; e < cnt; ++e) {
    const float4* src = reinterpret_cast<const float4*>(a.grad_pair + (size_t)(e0 + e) * kPairStride);
    const float4 u = src[0], w = src[1];
    const float z = src[2].x;
    G9[0] += u.x; G9[1] += u.y; G9[2] += u.z; G9[3] += u.w;
    G9[4] += w.x; G9[5] += w.y; G9[6] += w.z; G9[7] += w.w;
    G9[8] += z;
  }
  if (a.stat_grad) {  // densification statistics: view-space gradient norm of the visible Gaussian
    a.stat_grad[g] += sqrtf(G9[0] * G9[0] + G9[1] * G9[1]);
    a.stat_visible[g] += 1.f;
  }
  const CamParams& c = a.cam;
  const float4 co = a.conic_opacity[g];
  if (a.g_opacity) a.g_opacity[g] += G9[5] * co.w * (1.f - co.w);

  const float X0 = a.means[3 * g], X1 = a.means[3 * g + 1], X2 = a.means[3 * g + 2];
  float gX0 = 0.f, gX1 = 0.f, gX2 = 0.f;
  // ---- SH colour
  {
    const float cpx = -(c.m[0] * c.m[3] + c.m[4] * c.m[7] + c.m[8] * c.m[11]);
    const float cpy = -(c.m[1] * c.m[3] + c.m[5] * c.m[7] + c.m[9] * c.m[11]);
    const float cpz = -(c.m[2] * c.m[3] + c.m[6] * c.m[7] + c.m[10] * c.m[11]);
    const float vx = X0 - cpx, vy = X1 - cpy, vz = X2 - cpz;
    const float vn = sqrtf(vx * vx + vy * vy + vz * vz), vinv = 1.f / vn;
    const float dx = vx * vinv, dy = vy * vinv, dz = vz * vinv;
    float Y[16], dY[16][3];
    sh_basis_and_grad(a.sh_degree, dx, dy, dz, Y, dY);
    float gdir0 = 0.f, gdir1 = 0.f, gdir2 = 0.f;
    switch (a.sh_degree) {
      case 0: sh_colour_bwd<1>(a, g, Y, dY, G9, gdir0, gdir1, gdir2); break;
      case 1: sh_colour_bwd<4>(a, g, Y, dY, G9, gdir0, gdir1, gdir2); break;
      case 2: sh_colour_bwd<9>(a, g, Y, dY, G9, gdir0, gdir1, gdir2); break;
      default: sh_colour_bwd<16>(a, g, Y, dY, G9, gdir0, gdir1, gdir2); break;
    }
    const float dd = dx * gdir0 + dy * gdir1 + dz * gdir2;
    gX0 += (gdir0 - dx * dd) * vinv;
    gX1 += (gdir1 - dy * dd) * vinv;
    gX2 += (gdir2 - dz * dd) * vinv;
  }
  // ---- camera-space mean and the projected mean
  const float px = c.m[0] * X0 + c.m[1] * X1 + c.m[2] * X2 + c.m[3];
  const float py = c.m[4] * X0 + c.m[5] * X1 + c.m[6] * X2 + c.m[7];
  const float pz = c.m[8] * X0 + c.m[9] * X1 + c.m[10] * X2 + c.m[11];
  const float iz = 1.f / pz, iz2 = iz * iz;
  float gp0 = G9[0] * c.fx * iz, gp1 = G9[1] * c.fy * iz;
  float gp2 = -G9[0] * c.fx * px * iz2 - G9[1] * c.fy * py * iz2;
  // ---- conic = Sigma2D^-1: dL/dSigma2D = -K G_K K
  const float ka = co.x, kb = co.y, kc = co.z;
  const float gka = G9[2], gkb = 0.5f * G9[3], gkc = G9[4];
  // M = K G_K, then -M K
  const float m00 = ka * gka + kb * gkb, m01 = ka * gkb + kb * gkc;
  const float m10 = kb * gka + kc * gkb, m11 = kb * gkb + kc * gkc;
  const float S00 = -(m00 * ka + m01 * kb), S01 = -(m00 * kb + m01 * kc);
  const float S10 = -(m10 * ka + m11 * kb), S11 = -(m10 * kb + m11 * kc);
  // ---- Sigma2D = A A^T + 0.3 I, A = T R S, T = J W
  const float4 q4 = reinterpret_cast<const float4*>(a.quats)[g];
  const float qn = sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w), qinv = 1.f / qn;
  const float w = q4.x * qinv, x = q4.y * qinv, y = q4.z * qinv, z = q4.w * qinv;
  float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                   {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                   {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
  const float sc[3] = {expf(a.log_scales[3 * g]), expf(a.log_scales[3 * g + 1]), expf(a.log_scales[3 * g + 2])};
  const float limx = kGuard * (float)c.guard_w / (2.f * c.fx), limy = kGuard * (float)c.guard_h / (2.f * c.fy);
  const float rx_raw = px * iz, ry_raw = py * iz;
  const bool clx = fabsf(rx_raw) > limx, cly = fabsf(ry_raw) > limy;
  const float rx = fminf(limx, fmaxf(-limx, rx_raw)), ry = fminf(limy, fmaxf(-limy, ry_raw));
  const float J00 = c.fx * iz, J02 = -c.fx * rx * iz, J11 = c.fy * iz, J12 = -c.fy * ry * iz;
  float T[2][3] = {{J00 * c.m[0] + J02 * c.m[8], J00 * c.m[1] + J02 * c.m[9], J00 * c.m[2] + J02 * c.m[10]},
                   {J11 * c.m[4] + J12 * c.m[8], J11 * c.m[5] + J12 * c.m[9], J11 * c.m[6] + J12 * c.m[10]}};
  float RS[3][3], A[2][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) RS[i][j] = R[i][j] * sc[j];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) A[i][j] = T[i][0] * RS[0][j] + T[i][1] * RS[1][j] + T[i][2] * RS[2][j];
  // dL/dA = (S + S^T) A
  const float Ss00 = 2.f * S00, Ss01 = S01 + S10, Ss11 = 2.f * S11;
  float gA[2][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    gA[0][j] = Ss00 * A[0][j] + Ss01 * A[1][j];
    gA[1][j] = Ss01 * A[0][j] + Ss11 * A[1][j];
  }
  float gT[2][3], gRS[3][3];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) gT[i][j] = gA[i][0] * RS[j][0] + gA[i][1] * RS[j][1] + gA[i][2] * RS[j][2];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) gRS[i][j] = T[0][i] * gA[0][j] + T[1][i] * gA[1][j];
  float gR[3][3], gsc[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      gR[i][j] = gRS[i][j] * sc[j];
      gsc[j] += gRS[i][j] * R[i][j];
    }
  // dR/dq for the unit quaternion (w, x, y, z)
  const float gw = 2.f * (-z * gR[0][1] + y * gR[0][2] + z * gR[1][0] - x * gR[1][2] - y * gR[2][0] + x * gR[2][1]);
  const float gx = 2.f * (y * gR[0][1] + z * gR[0][2] + y * gR[1][0] - w * gR[1][2] + z * gR[2][0] + w * gR[2][1]) -
                   4.f * x * (gR[1][1] + gR[2][2]);
  const float gy = 2.f * (x * gR[0][1] + w * gR[0][2] + x * gR[1][0] + z * gR[1][2] - w * gR[2][0] + z * gR[2][1]) -
                   4.f * y * (gR[0][0] + gR[2][2]);
  const float gz = 2.f * (-w * gR[0][1] + x * gR[0][2] + w * gR[1][0] + y * gR[1][2] + x * gR[2][0] + y * gR[2][1]) -
                   4.f * z * (gR[0][0] + gR[1][1]);
  const float qd = w * gw + x * gx + y * gy + z * gz;
  // T = J W: dL/dJ = dL/dT W^T (only the non-zero entries of J matter)
  const float gJ00 = gT[0][0] * c.m[0] + gT[0][1] * c.m[1] + gT[0][2] * c.m[2];
  const float gJ02 = gT[0][0] * c.m[8] + gT[0][1] * c.m[9] + gT[0][2] * c.m[10];
  const float gJ11 = gT[1][0] * c.m[4] + gT[1][1] * c.m[5] + gT[1][2] * c.m[6];
  const float gJ12 = gT[1][0] * c.m[8] + gT[1][1] * c.m[9] + gT[1][2] * c.m[10];
  gp2 += -gJ00 * c.fx * iz2 - gJ11 * c.fy * iz2;
  if (!clx) {
    gp0 += -gJ02 * c.fx * iz2;
    gp2 += gJ02 * 2.f * c.fx * px * iz2 * iz;
  } else {
    gp2 += gJ02 * c.fx * rx * iz2;
  }
  if (!cly) {
    gp1 += -gJ12 * c.fy * iz2;
    gp2 += gJ12 * 2.f * c.fy * py * iz2 * iz;
  } else {
    gp2 += gJ12 * c.fy * ry * iz2;
  }
  gX0 += c.m[0] * gp0 + c.m[4] * gp1 + c.m[8] * gp2;
  gX1 += c.m[1] * gp0 + c.m[5] * gp1 + c.m[9] * gp2;
  gX2 += c.m[2] * gp0 + c.m[6] * gp1 + c.m[10] * gp2;
  const float gq[4] = {(gw - w * qd) * qinv, (gx - x * qd) * qinv, (gy - y * qd) * qinv, (gz - z * qd) * qinv};
  const float gs[3] = {gsc[0] * sc[0], gsc[1] * sc[1], gsc[2] * sc[2]};
  gd[0] = gX0; gd[1] = gX1; gd[2] = gX2;
  gd[3] = gq[0]; gd[4] = gq[1]; gd[5] = gq[2]; gd[6] = gq[3];
  gd[7] = gs[0]; gd[8] = gs[1]; gd[9] = gs[2];
  if (a.g_means) {
    a.g_means[3 * g] += gX0; a.g_means[3 * g + 1] += gX1; a.g_means[3 * g + 2] += gX2;
  }
  if (a.g_quats)
#pragma unroll
    for (int k = 0; k < 4; ++k) a.g_quats[4 * g + k] += gq[k];
  if (a.g_log_scales)
#pragma unroll
    for (int k = 0; k < 3; ++k) a.g_log_scales[3 * g + k] += gs[k];
}

// ------------------------------------------------------------------ MLP + HexPlane

// Threads of the MLP backward CTA (one CTA per SM: the weights and the activation
// columns fill shared memory): 256 where they fit, else 128.
constexpr int kMTMax = 256;

__device__ __forceinline__ void axis_setup(float u, int R, int& i0, float& f, float& dfdu) {
  const float uc = fminf(1.f, fmaxf(-1.f, u));
  const float g = (uc + 1.f) * 0.5f * (float)(R - 1);
  int i = (int)floorf(g);
  i = max(0, min(i, R - 2));
  i0 = i;
  f = g - (float)i;
  dfdu = (u > -1.f && u < 1.f) ? 0.5f * (float)(R - 1) : 0.f;
}

// y = b + Wt^T x over IN inputs read from this thread's shared-memory column.
template <int IN, int MT>
__device__ __forceinline__ void dense64(const float* __restrict__ Wt, const float* __restrict__ b,
                                        const float* __restrict__ col, float (&y)[kWidth]) {
#pragma unroll
  for (int o = 0; o < kWidth; ++o) y[o] = b[o];
#pragma unroll 2
  for (int i = 0; i < IN; ++i) {
    const float x = col[i * MT];
    const float4* w4 = reinterpret_cast<const float4*>(Wt + i * kWidth);
#pragma unroll
    for (int q = 0; q < kWidth / 4; ++q) {
      const float4 ww = w4[q];
      y[4 * q + 0] = fmaf(ww.x, x, y[4 * q + 0]);
      y[4 * q + 1] = fmaf(ww.y, x, y[4 * q + 1]);
      y[4 * q + 2] = fmaf(ww.z, x, y[4 * q + 2]);
      y[4 * q + 3] = fmaf(ww.w, x, y[4 * q + 3]);
    }
  }
}

// gcol[i] (+)= sum_o Wt[i][o] d[o] for i < IN.
template <int IN, bool ACC, int MT>
__device__ __forceinline__ void dense64_bwd(const float* __restrict__ Wt, const float (&d)[kWidth], float* gcol) {
#pragma unroll 2
  for (int i = 0; i < IN; ++i) {
    const float4* w4 = reinterpret_cast<const float4*>(Wt + i * kWidth);
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < kWidth / 4; ++q) {
      const float4 ww = w4[q];
      s = fmaf(ww.x, d[4 * q], s);
      s = fmaf(ww.y, d[4 * q + 1], s);
      s = fmaf(ww.z, d[4 * q + 2], s);
      s = fmaf(ww.w, d[4 * q + 3], s);
    }
    gcol[i * MT] = ACC ? gcol[i * MT] + s : s;
  }
}

template <int OUT, int MT>
__device__ __forceinline__ void head_bwd(const float* __restrict__ sw, const MlpGeomT& mg, int layer, float* col,
                                         float* gcol, const float* dout, float* hid_out, float* dh_out,
                                         long long n, long long g) {
  float y[kWidth];
  dense64<kWidth, MT>(sw + mg.w[layer], sw + mg.b[layer], col, y);
  const float* W2 = sw + mg.w[layer + 1];  // [64][OUT]
  float d[kWidth];
#pragma unroll
  for (int o = 0; o < kWidth; ++o) {
    hid_out[(long long)o * n + g] = fmaxf(y[o], 0.f);
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < OUT; ++j) s = fmaf(W2[o * OUT + j], dout[j], s);
    d[o] = y[o] > 0.f ? s : 0.f;
    dh_out[(long long)o * n + g] = d[o];
  }
  dense64_bwd<kWidth, true, MT>(sw + mg.w[layer], d, gcol);
}

template <int H, int L, int MT>
__global__ void __launch_bounds__(MT, 1) mlp_bwd_kernel(MlpBwdArgs a) {
  constexpr int HL = H * L;
  constexpr int ROWS = HL > kWidth ? HL : kWidth;
  extern __shared__ float4 smem4[];
  const DeformArgs& f = a.f;
  float* sw = reinterpret_cast<float*>(smem4);
  float* colbase = sw + f.mg.total;
  float* gcolbase = colbase + ROWS * MT;
  for (int i = threadIdx.x; i < f.mg.total / 4; i += MT)
    smem4[i] = __ldg(reinterpret_cast<const float4*>(f.mlp_t) + i);
  __syncthreads();
  const PlaneGeom& pg = f.pg;
  float* col = colbase + threadIdx.x;
  float* gcol = gcolbase + threadIdx.x;
  const long long n = f.n;
  const MlpActs& act = a.act;
  // Gaussians in the scene's Morton work order (neighbouring plane cells for the
  // taps and the gradient atomics of one warp); the activation columns are kept in
  // that order too (the weight-gradient sums do not depend on the column order)
  for (long long ii = (long long)blockIdx.x * MT + threadIdx.x; ii < n; ii += (long long)gridDim.x * MT) {
    const long long g = f.perm ? (long long)f.perm[ii] : ii;
    const float X[3] = {f.means[3 * g], f.means[3 * g + 1], f.means[3 * g + 2]};
    float c[4], dcdx[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      c[k] = (X[k] - pg.aabb_min[k]) * pg.aabb_scale[k] - 1.f;
      dcdx[k] = pg.aabb_scale[k];
    }
    c[3] = 2.f * f.t0 - 1.f;
    // ---- forward recompute (Eq. 5, phi_d)
#pragma unroll
    for (int l = 0; l < L; ++l) {
      float fv[H];
#pragma unroll
      for (int k = 0; k < H; ++k) fv[k] = 1.f;
#pragma unroll
      for (int p = 0; p < 6; ++p) {
        const int ax = (p < 2) ? 0 : (p == 2 ? 1 : p - 3);
        const int bx = (p == 0) ? 1 : (p <= 2 ? 2 : 3);
        const int Ra = ax < 3 ? pg.res[l] : pg.res_time, Rb = bx < 3 ? pg.res[l] : pg.res_time;
        int i0, j0;
        float fa, fb, da, db;
        axis_setup(c[ax], Ra, i0, fa, da);
        axis_setup(c[bx], Rb, j0, fb, db);
        const float4* v00 = reinterpret_cast<const float4*>(f.planes + pg.off[l][p] + ((long long)j0 * Ra + i0) * H);
        const float4* v10 = v00 + H / 4;
        const float4* v01 = v00 + (long long)Ra * (H / 4);
        const float4* v11 = v01 + H / 4;
        const float w00 = (1.f - fa) * (1.f - fb), w10 = fa * (1.f - fb), w01 = (1.f - fa) * fb, w11 = fa * fb;
#pragma unroll
        for (int q = 0; q < H / 4; ++q) {
          const float4 A = __ldg(v00 + q), B = __ldg(v10 + q), C = __ldg(v01 + q), D = __ldg(v11 + q);
          fv[4 * q + 0] *= w00 * A.x + w10 * B.x + w01 * C.x + w11 * D.x;
          fv[4 * q + 1] *= w00 * A.y + w10 * B.y + w01 * C.y + w11 * D.y;
          fv[4 * q + 2] *= w00 * A.z + w10 * B.z + w01 * C.z + w11 * D.z;
          fv[4 * q + 3] *= w00 * A.w + w10 * B.w + w01 * C.w + w11 * D.w;
        }
      }
#pragma unroll
      for (int k = 0; k < H; ++k) {
        col[(l * H + k) * MT] = fv[k];
        act.fh[(long long)(l * H + k) * n + ii] = fv[k];
      }
    }
    float y[kWidth];
    dense64<HL, MT>(sw + f.mg.w[0], sw + f.mg.b[0], col, y);
#pragma unroll
    for (int o = 0; o < kWidth; ++o) {
      const float v = fmaxf(y[o], 0.f);
      act.a1[(long long)o * n + ii] = v;
      col[o * MT] = v;
    }
    dense64<kWidth, MT>(sw + f.mg.w[1], sw + f.mg.b[1], col, y);
#pragma unroll
    for (int o = 0; o < kWidth; ++o) {
      const float v = fmaxf(y[o], 0.f);
      act.fd[(long long)o * n + ii] = v;
      col[o * MT] = v;
    }
    // ---- heads backward (output deltas = dL/d(X', r', s'), Eq. 6)
    float dout[kDeltaDim];
#pragma unroll
    for (int j = 0; j < kDeltaDim; ++j) {
      dout[j] = a.gd[10 * g + j];
      act.dout[(long long)j * n + ii] = dout[j];
    }
#pragma unroll
    for (int i = 0; i < kWidth; ++i) gcol[i * MT] = 0.f;
    head_bwd<3, MT>(sw, f.mg, 2, col, gcol, dout, act.hid, act.dh, n, ii);
    head_bwd<4, MT>(sw, f.mg, 4, col, gcol, dout + 3, act.hid + 64 * n, act.dh + 64 * n, n, ii);
    head_bwd<3, MT>(sw, f.mg, 6, col, gcol, dout + 7, act.hid + 128 * n, act.dh + 128 * n, n, ii);
    // ---- phi_d backward
    float d[kWidth];
#pragma unroll
    for (int o = 0; o < kWidth; ++o) {
      d[o] = col[o * MT] > 0.f ? gcol[o * MT] : 0.f;
      act.d2[(long long)o * n + ii] = d[o];
    }
    dense64_bwd<kWidth, false, MT>(sw + f.mg.w[1], d, gcol);
#pragma unroll
    for (int o = 0; o < kWidth; ++o) {
      d[o] = act.a1[(long long)o * n + ii] > 0.f ? gcol[o * MT] : 0.f;
      act.d1[(long long)o * n + ii] = d[o];
    }
    dense64_bwd<HL, false, MT>(sw + f.mg.w[0], d, gcol);  // gcol[0..HL) = dL/df_h
    // ---- Eq. 5 backward: plane cells and the sampling position
    float gx[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
    for (int l = 0; l < L; ++l) {
      float v[6][H];
      int i0[6], j0[6], Ra[6];
      float fa[6], fb[6], da[6], db[6];
#pragma unroll
      for (int p = 0; p < 6; ++p) {
        const int ax = (p < 2) ? 0 : (p == 2 ? 1 : p - 3);
        const int bx = (p == 0) ? 1 : (p <= 2 ? 2 : 3);
        Ra[p] = ax < 3 ? pg.res[l] : pg.res_time;
        const int Rb = bx < 3 ? pg.res[l] : pg.res_time;
        axis_setup(c[ax], Ra[p], i0[p], fa[p], da[p]);
        axis_setup(c[bx], Rb, j0[p], fb[p], db[p]);
        const float* P = f.planes + pg.off[l][p] + ((long long)j0[p] * Ra[p] + i0[p]) * H;
        const float w00 = (1.f - fa[p]) * (1.f - fb[p]), w10 = fa[p] * (1.f - fb[p]),
                    w01 = (1.f - fa[p]) * fb[p], w11 = fa[p] * fb[p];
#pragma unroll
        for (int k = 0; k < H; ++k)
          v[p][k] = w00 * __ldg(P + k) + w10 * __ldg(P + H + k) + w01 * __ldg(P + (long long)Ra[p] * H + k) +
                    w11 * __ldg(P + (long long)Ra[p] * H + H + k);
      }
#pragma unroll
      for (int p = 0; p < 6; ++p) {
        const int ax = (p < 2) ? 0 : (p == 2 ? 1 : p - 3);
        const int bx = (p == 0) ? 1 : (p <= 2 ? 2 : 3);
        const float* P = f.planes + pg.off[l][p] + ((long long)j0[p] * Ra[p] + i0[p]) * H;
        float* GP = a.g_planes ? a.g_planes + pg.off[l][p] + ((long long)j0[p] * Ra[p] + i0[p]) * H : nullptr;
        const float w00 = (1.f - fa[p]) * (1.f - fb[p]), w10 = fa[p] * (1.f - fb[p]),
                    w01 = (1.f - fa[p]) * fb[p], w11 = fa[p] * fb[p];
        float sa = 0.f, sb = 0.f;
#pragma unroll
        for (int q = 0; q < H / 4; ++q) {
          float gv[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int k = 4 * q + e;
            float others = 1.f;
#pragma unroll
            for (int r = 0; r < 6; ++r)
              if (r != p) others *= v[r][k];
            gv[e] = gcol[(l * H + k) * MT] * others;
            const float p00 = __ldg(P + k), p10 = __ldg(P + H + k), p01 = __ldg(P + (long long)Ra[p] * H + k),
                        p11 = __ldg(P + (long long)Ra[p] * H + H + k);
            sa += gv[e] * ((1.f - fb[p]) * (p10 - p00) + fb[p] * (p11 - p01));
            sb += gv[e] * ((1.f - fa[p]) * (p01 - p00) + fa[p] * (p11 - p10));
          }
          if (GP) {
            atomicAdd(reinterpret_cast<float4*>(GP) + q, make_float4(w00 * gv[0], w00 * gv[1], w00 * gv[2], w00 * gv[3]));
            atomicAdd(reinterpret_cast<float4*>(GP + H) + q,
                      make_float4(w10 * gv[0], w10 * gv[1], w10 * gv[2], w10 * gv[3]));
            atomicAdd(reinterpret_cast<float4*>(GP + (long long)Ra[p] * H) + q,
                      make_float4(w01 * gv[0], w01 * gv[1], w01 * gv[2], w01 * gv[3]));
            atomicAdd(reinterpret_cast<float4*>(GP + (long long)Ra[p] * H + H) + q,
                      make_float4(w11 * gv[0], w11 * gv[1], w11 * gv[2], w11 * gv[3]));
          }
        }
        if (ax < 3) gx[ax] += sa * da[p] * dcdx[ax];
        if (bx < 3) gx[bx] += sb * db[p] * dcdx[bx];
      }
    }
    if (a.g_means) {
      a.g_means[3 * g] += gx[0];
      a.g_means[3 * g + 1] += gx[1];
      a.g_means[3 * g + 2] += gx[2];
    }
  }
}

template <int H, int L, int MT>
cudaError_t launch_mlp_mt(const MlpBwdArgs& a, size_t smem, cudaStream_t s) {
  static PerDeviceFlag attr;
  cudaError_t e = once_per_device(attr, [&] {
    return cudaFuncSetAttribute(mlp_bwd_kernel<H, L, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
  const int sms = device_sm_count();
  const long long need = ((long long)a.f.n + MT - 1) / MT;
  const int grid = (int)(need < sms ? need : sms);
  mlp_bwd_kernel<H, L, MT><<<grid, MT, smem, s>>>(a);
  return cudaGetLastError();
}

template <int H, int L>
cudaError_t launch_mlp_t(const MlpBwdArgs& a, cudaStream_t s) {
  constexpr int HL = H * L;
  constexpr int rows = HL > kWidth ? HL : kWidth;
  const size_t big = sizeof(float) * ((size_t)a.f.mg.total + 2 * (size_t)rows * kMTMax);
  if (big <= 227 * 1024) return launch_mlp_mt<H, L, kMTMax>(a, big, s);
  return launch_mlp_mt<H, L, kMTMax / 2>(a, sizeof(float) * ((size_t)a.f.mg.total + 2 * (size_t)rows * (kMTMax / 2)),
                                        s);
}

// ------------------------------------------------------------------ MLP + HexPlane, tiled
// The same backward over tiles of 64 Gaussians (Morton work order), every layer
// a register-blocked SIMT GEMM over activations held feature-major in shared
// memory ([feature][68]): thread (tid & 15, tid >> 4) owns Gaussians 4(tid & 15)..+3
// and outputs 4(tid >> 4)..+3, so two 128-bit shared loads feed 16 FMAs in the
// forward layers (Wt[in][out] rows) and one 128-bit + four broadcast scalar loads
// in the transposed backward layers.  The deltas overwrite the activations they
// are masked by (ReLU'), and every activation/delta the weight gradients need is
// copied out to the feature-major global arrays with coalesced stores.
constexpr int kTT = 256;          // threads
constexpr int kTG = 64;           // Gaussians per tile
constexpr int kTS = kTG + 4;      // row stride (floats) of the shared activation arrays

// acc[g][o] = b[o4 + o] + sum_i Wt[i][o4 + o] src[i][g4 + g]
template <int IN>
__device__ __forceinline__ void t_fwd(const float* __restrict__ Wt, int ldw, const float* __restrict__ b,
                                      const float* __restrict__ src, int g4, int o4, float (&acc)[4][4]) {
#pragma unroll
  for (int o = 0; o < 4; ++o)
#pragma unroll
    for (int g = 0; g < 4; ++g) acc[g][o] = b[o4 + o];
  float2 a2[4][2];  // outputs in pairs: one f32x2 FMA per two (each element the same FP32 FMA)
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    a2[g][0] = make_float2(acc[g][0], acc[g][1]);
    a2[g][1] = make_float2(acc[g][2], acc[g][3]);
  }
#pragma unroll 4
  for (int i = 0; i < IN; ++i) {
    const float4 x = *reinterpret_cast<const float4*>(src + i * kTS + g4);
    const float4 w = *reinterpret_cast<const float4*>(Wt + i * ldw + o4);
    const float xs[4] = {x.x, x.y, x.z, x.w};
    const float2 w01 = make_float2(w.x, w.y), w23 = make_float2(w.z, w.w);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const float2 xg = make_float2(xs[g], xs[g]);
      a2[g][0] = __ffma2_rn(w01, xg, a2[g][0]);
      a2[g][1] = __ffma2_rn(w23, xg, a2[g][1]);
    }
  }
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    acc[g][0] = a2[g][0].x; acc[g][1] = a2[g][0].y;
    acc[g][2] = a2[g][1].x; acc[g][3] = a2[g][1].y;
  }
}

// acc[g][i] += sum_{o < nout} Wt[(i4 + i) * ldw + o] d[o][g4 + g]  (the transposed layer)
__device__ __forceinline__ void t_bwd(const float* __restrict__ Wt, int ldw, const float* __restrict__ d, int nout,
                                      int g4, int i4, float (&acc)[4][4]) {
  float2 a2[4][2];  // inputs in pairs: one f32x2 FMA per two (each element the same FP32 FMA)
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    a2[g][0] = make_float2(acc[g][0], acc[g][1]);
    a2[g][1] = make_float2(acc[g][2], acc[g][3]);
  }
#pragma unroll 4
  for (int o = 0; o < nout; ++o) {
    const float4 x = *reinterpret_cast<const float4*>(d + o * kTS + g4);
    const float2 w01 = make_float2(Wt[(i4 + 0) * ldw + o], Wt[(i4 + 1) * ldw + o]),
                 w23 = make_float2(Wt[(i4 + 2) * ldw + o], Wt[(i4 + 3) * ldw + o]);
    const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const float2 xg = make_float2(xs[g], xs[g]);
      a2[g][0] = __ffma2_rn(w01, xg, a2[g][0]);
      a2[g][1] = __ffma2_rn(w23, xg, a2[g][1]);
    }
  }
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    acc[g][0] = a2[g][0].x; acc[g][1] = a2[g][0].y;
    acc[g][2] = a2[g][1].x; acc[g][3] = a2[g][1].y;
  }
}

__device__ __forceinline__ void t_store(float* dst, int g4, int o4, const float (&acc)[4][4], bool relu) {
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    float4 v = make_float4(acc[0][o], acc[1][o], acc[2][o], acc[3][o]);
    if (relu) v = make_float4(fmaxf(v.x, 0.f), fmaxf(v.y, 0.f), fmaxf(v.z, 0.f), fmaxf(v.w, 0.f));
    *reinterpret_cast<float4*>(dst + (o4 + o) * kTS + g4) = v;
  }
}

// dst = acc where the activation `act` (same element) is positive, else 0 (ReLU'), in place
__device__ __forceinline__ void t_store_masked(float* dst, int g4, int o4, const float (&acc)[4][4]) {
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    float4* p = reinterpret_cast<float4*>(dst + (o4 + o) * kTS + g4);
    const float4 a = *p;
    *p = make_float4(a.x > 0.f ? acc[0][o] : 0.f, a.y > 0.f ? acc[1][o] : 0.f, a.z > 0.f ? acc[2][o] : 0.f,
                     a.w > 0.f ? acc[3][o] : 0.f);
  }
}

// rows [0, rows) of a shared [rows][kTS] array to global [rows][n] at columns base.. (m valid)
__device__ __forceinline__ void t_copy_out(const float* src, int rows, float* dst, long long n, long long base,
                                           int m) {
  for (int e = threadIdx.x; e < rows * kTG; e += kTT) {
    const int r = e / kTG, c = e % kTG;
    if (c < m) dst[(long long)r * n + base + c] = src[r * kTS + c];
  }
}

template <int H, int L>
__global__ void __launch_bounds__(kTT, 1) mlp_bwd_tile_kernel(MlpBwdArgs a) {
  constexpr int HL = H * L;
  constexpr int Q = H / 4;
  extern __shared__ float4 smem4[];
  const DeformArgs& f = a.f;
  const MlpGeomT& mg = f.mg;
  const PlaneGeom& pg = f.pg;
  float* sw = reinterpret_cast<float*>(smem4);
  float* FH = sw + mg.total;          // [HL][kTS]: f_h, later dL/df_h
  float* A1 = FH + HL * kTS;          // [64]: a1, later its delta
  float* FD = A1 + kWidth * kTS;      // [64]: f_d, later its delta
  float* HID = FD + kWidth * kTS;     // [192]: head hidden activations, later their deltas
  float* DO = HID + 3 * kWidth * kTS; // [10]: dL/d(X', r', s')
  float4* sRow = reinterpret_cast<float4*>(DO + kDeltaDim * kTS);  // (X, t) per Gaussian
  int* sG = reinterpret_cast<int*>(sRow + kTG);                     // Gaussian index per column
  // the weights by cp.async (every 16-byte copy in flight at once), waited for below
  for (int i = threadIdx.x; i < mg.total / 4; i += kTT) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem4 + i);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(reinterpret_cast<const float4*>(f.mlp_t) + i)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;\n" "cp.async.wait_all;\n" ::: "memory");
  const int g4 = (threadIdx.x & 15) * 4, o4 = (threadIdx.x >> 4) * 4;
  const long long n = f.n;
  const MlpActs& act = a.act;
  const long long tiles = (n + kTG - 1) / kTG;
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long long base = tile * kTG;
    const int m = (int)min((long long)kTG, n - base);
    __syncthreads();  // weights loaded / the previous tile done with every array
    if (threadIdx.x < kTG) {
      const int r = threadIdx.x;
      float4 x = make_float4(0.f, 0.f, 0.f, f.t0);
      int g = -1;
      if (r < m) {
        g = f.perm ? (int)f.perm[base + r] : (int)(base + r);
        x = make_float4(f.means[3 * g], f.means[3 * g + 1], f.means[3 * g + 2], f.t0);
      }
      sRow[r] = x;
      sG[r] = g;
      for (int j = 0; j < kDeltaDim; ++j) DO[j * kTS + r] = g >= 0 ? a.gd[10 * (long long)g + j] : 0.f;
    }
    __syncthreads();
    // ---- Eq. 5 recompute: f_h (lane-cooperative: Q lanes per (Gaussian, level), a float4 each)
    for (int item = threadIdx.x; item < kTG * L * Q; item += kTT) {
      const int q = item % Q, rl = item / Q, r = rl % kTG, l = rl / kTG;
      float fv[4] = {0.f, 0.f, 0.f, 0.f};
      if (r < m) {
        const float4 xr = sRow[r];
        const float c[4] = {(xr.x - pg.aabb_min[0]) * pg.aabb_scale[0] - 1.f,
                            (xr.y - pg.aabb_min[1]) * pg.aabb_scale[1] - 1.f,
                            (xr.z - pg.aabb_min[2]) * pg.aabb_scale[2] - 1.f, 2.f * xr.w - 1.f};
        fv[0] = fv[1] = fv[2] = fv[3] = 1.f;
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          const int ax = (p < 2) ? 0 : (p == 2 ? 1 : p - 3);
          const int bx = (p == 0) ? 1 : (p <= 2 ? 2 : 3);
          const int Ra = ax < 3 ? pg.res[l] : pg.res_time, Rb = bx < 3 ? pg.res[l] : pg.res_time;
          int i0, j0;
          float fa, fb, da, db;
          axis_setup(c[ax], Ra, i0, fa, da);
          axis_setup(c[bx], Rb, j0, fb, db);
          const float4* v00 =
              reinterpret_cast<const float4*>(f.planes + pg.off[l][p] + ((long long)j0 * Ra + i0) * H) + q;
          const float4 A = __ldg(v00), B = __ldg(v00 + Q), C = __ldg(v00 + (long long)Ra * Q),
                       D = __ldg(v00 + (long long)Ra * Q + Q);
          const float w00 = (1.f - fa) * (1.f - fb), w10 = fa * (1.f - fb), w01 = (1.f - fa) * fb, w11 = fa * fb;
          fv[0] *= w00 * A.x + w10 * B.x + w01 * C.x + w11 * D.x;
          fv[1] *= w00 * A.y + w10 * B.y + w01 * C.y + w11 * D.y;
          fv[2] *= w00 * A.z + w10 * B.z + w01 * C.z + w11 * D.z;
          fv[3] *= w00 * A.w + w10 * B.w + w01 * C.w + w11 * D.w;
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) FH[(l * H + 4 * q + e) * kTS + r] = fv[e];
    }
    __syncthreads();
    t_copy_out(FH, HL, act.fh, n, base, m);
    t_copy_out(DO, kDeltaDim, act.dout, n, base, m);
    // ---- forward recompute: a1, f_d, head hidden layers
    float acc[4][4];
    if (o4 < kWidth) {
      t_fwd<HL>(sw + mg.w[0], kWidth, sw + mg.b[0], FH, g4, o4, acc);
      t_store(A1, g4, o4, acc, true);
    }
    __syncthreads();
    t_copy_out(A1, kWidth, act.a1, n, base, m);
    t_fwd<kWidth>(sw + mg.w[1], kWidth, sw + mg.b[1], A1, g4, o4, acc);
    t_store(FD, g4, o4, acc, true);
    __syncthreads();
    t_copy_out(FD, kWidth, act.fd, n, base, m);
#pragma unroll 1
    for (int h = 0; h < 3; ++h) {
      t_fwd<kWidth>(sw + mg.w[2 + 2 * h], kWidth, sw + mg.b[2 + 2 * h], FD, g4, o4, acc);
      t_store(HID + kWidth * h * kTS, g4, o4, acc, true);
    }
    __syncthreads();
    t_copy_out(HID, 3 * kWidth, act.hid, n, base, m);
    // ---- heads: d_hid = ReLU'(hid) (W_out^T dL/d(X', r', s')), in place over HID
    {
      const int col0[3] = {0, 3, 7}, outs[3] = {3, 4, 3};
      for (int e = threadIdx.x; e < 3 * kWidth * kTG; e += kTT) {
        const int r = e % kTG, ho = e / kTG, h = ho / kWidth, o = ho % kWidth;
        const float* W2 = sw + mg.w[3 + 2 * h];  // Wt[o][j]
        float sacc = 0.f;
        for (int j = 0; j < outs[h]; ++j) sacc = fmaf(W2[o * outs[h] + j], DO[(col0[h] + j) * kTS + r], sacc);
        float& hv = HID[ho * kTS + r];
        hv = hv > 0.f ? sacc : 0.f;
      }
    }
    __syncthreads();
    t_copy_out(HID, 3 * kWidth, act.dh, n, base, m);
    // ---- phi_d: d_fd = ReLU'(f_d) sum_h W_h1^T d_hid_h, in place over FD
#pragma unroll
    for (int g = 0; g < 4; ++g)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[g][i] = 0.f;
#pragma unroll 1
    for (int h = 0; h < 3; ++h) t_bwd(sw + mg.w[2 + 2 * h], kWidth, HID + kWidth * h * kTS, kWidth, g4, o4, acc);
    t_store_masked(FD, g4, o4, acc);
    __syncthreads();
    t_copy_out(FD, kWidth, act.d2, n, base, m);
    // d_a1 = ReLU'(a1) W2^T d_fd, in place over A1
#pragma unroll
    for (int g = 0; g < 4; ++g)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[g][i] = 0.f;
    t_bwd(sw + mg.w[1], kWidth, FD, kWidth, g4, o4, acc);
    t_store_masked(A1, g4, o4, acc);
    __syncthreads();
    t_copy_out(A1, kWidth, act.d1, n, base, m);
    // dL/df_h = W1^T d_a1 (HL rows, 64 per pass), over FH
#pragma unroll 1
    for (int i0 = 0; i0 < HL; i0 += kWidth) {
      if (i0 + o4 < HL) {
#pragma unroll
        for (int g = 0; g < 4; ++g)
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[g][i] = 0.f;
        t_bwd(sw + mg.w[0] + (long long)i0 * kWidth, kWidth, A1, kWidth, g4, o4, acc);
        t_store(FH + i0 * kTS, g4, o4, acc, false);
      }
    }
    __syncthreads();
    // ---- Eq. 5 backward: plane cells (float4 atomics) and the sampling position
    for (int item = threadIdx.x; item < kTG * L * Q; item += kTT) {
      const int q = item % Q, rl = item / Q, r = rl % kTG, l = rl / kTG;
      const bool live = r < m;
      float gxs[3] = {0.f, 0.f, 0.f};
      if (live) {
        const float4 xr = sRow[r];
        const float c[4] = {(xr.x - pg.aabb_min[0]) * pg.aabb_scale[0] - 1.f,
                            (xr.y - pg.aabb_min[1]) * pg.aabb_scale[1] - 1.f,
                            (xr.z - pg.aabb_min[2]) * pg.aabb_scale[2] - 1.f, 2.f * xr.w - 1.f};
        float v[6][4];
        int i0s[6], j0s[6], Ras[6];
        float fas[6], fbs[6], das[6], dbs[6];
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          const int ax = (p < 2) ? 0 : (p == 2 ? 1 : p - 3);
          const int bx = (p == 0) ? 1 : (p <= 2 ? 2 : 3);
          Ras[p] = ax < 3 ? pg.res[l] : pg.res_time;
          const int Rb = bx < 3 ? pg.res[l] : pg.res_time;
          axis_setup(c[ax], Ras[p], i0s[p], fas[p], das[p]);
          axis_setup(c[bx], Rb, j0s[p], fbs[p], dbs[p]);
          const float4* v00 =
              reinterpret_cast<const float4*>(f.planes + pg.off[l][p] + ((long long)j0s[p] * Ras[p] + i0s[p]) * H) + q;
          const float4 A = __ldg(v00), B = __ldg(v00 + Q), C = __ldg(v00 + (long long)Ras[p] * Q),
                       D = __ldg(v00 + (long long)Ras[p] * Q + Q);
          const float w00 = (1.f - fas[p]) * (1.f - fbs[p]), w10 = fas[p] * (1.f - fbs[p]),
                      w01 = (1.f - fas[p]) * fbs[p], w11 = fas[p] * fbs[p];
          v[p][0] = w00 * A.x + w10 * B.x + w01 * C.x + w11 * D.x;
          v[p][1] = w00 * A.y + w10 * B.y + w01 * C.y + w11 * D.y;
          v[p][2] = w00 * A.z + w10 * B.z + w01 * C.z + w11 * D.z;
          v[p][3] = w00 * A.w + w10 * B.w + w01 * C.w + w11 * D.w;
        }
        float gf[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) gf[e] = FH[(l * H + 4 * q + e) * kTS + r];
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          const int ax = (p < 2) ? 0 : (p == 2 ? 1 : p - 3);
          const int bx = (p == 0) ? 1 : (p <= 2 ? 2 : 3);
          float gv[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            float others = 1.f;
#pragma unroll
            for (int r2 = 0; r2 < 6; ++r2)
              if (r2 != p) others *= v[r2][e];
            gv[e] = gf[e] * others;
          }
          const long long cell = pg.off[l][p] + ((long long)j0s[p] * Ras[p] + i0s[p]) * H + 4 * q;
          const float* P = f.planes + cell;
          const float4 A = __ldg(reinterpret_cast<const float4*>(P)), B = __ldg(reinterpret_cast<const float4*>(P + H)),
                       C = __ldg(reinterpret_cast<const float4*>(P + (long long)Ras[p] * H)),
                       D = __ldg(reinterpret_cast<const float4*>(P + (long long)Ras[p] * H + H));
          const float fa = fas[p], fb = fbs[p];
          const float As[4] = {A.x, A.y, A.z, A.w}, Bs[4] = {B.x, B.y, B.z, B.w}, Cs[4] = {C.x, C.y, C.z, C.w},
                      Ds[4] = {D.x, D.y, D.z, D.w};
          float sa = 0.f, sb = 0.f;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            sa += gv[e] * ((1.f - fb) * (Bs[e] - As[e]) + fb * (Ds[e] - Cs[e]));
            sb += gv[e] * ((1.f - fa) * (Cs[e] - As[e]) + fa * (Ds[e] - Bs[e]));
          }
          if (a.g_planes) {
            float* GP = a.g_planes + cell;
            const float w00 = (1.f - fa) * (1.f - fb), w10 = fa * (1.f - fb), w01 = (1.f - fa) * fb, w11 = fa * fb;
            atomicAdd(reinterpret_cast<float4*>(GP), make_float4(w00 * gv[0], w00 * gv[1], w00 * gv[2], w00 * gv[3]));
            atomicAdd(reinterpret_cast<float4*>(GP + H),
                      make_float4(w10 * gv[0], w10 * gv[1], w10 * gv[2], w10 * gv[3]));
            atomicAdd(reinterpret_cast<float4*>(GP + (long long)Ras[p] * H),
                      make_float4(w01 * gv[0], w01 * gv[1], w01 * gv[2], w01 * gv[3]));
            atomicAdd(reinterpret_cast<float4*>(GP + (long long)Ras[p] * H + H),
                      make_float4(w11 * gv[0], w11 * gv[1], w11 * gv[2], w11 * gv[3]));
          }
          if (ax < 3) gxs[ax] += sa * das[p] * pg.aabb_scale[ax];
          if (bx < 3) gxs[bx] += sb * dbs[p] * pg.aabb_scale[bx];
        }
      }
      // the Q lanes of one (Gaussian, level) are consecutive and Q divides 32
#pragma unroll
      for (int w = 1; w < Q; w <<= 1)
#pragma unroll
        for (int k = 0; k < 3; ++k) gxs[k] += __shfl_xor_sync(0xffffffffu, gxs[k], w);
      if (live && q == 0 && a.g_means) {
        const int g = sG[r];
        // levels of one Gaussian are different items: accumulate atomically
        atomicAdd(&a.g_means[3 * (long long)g], gxs[0]);
        atomicAdd(&a.g_means[3 * (long long)g + 1], gxs[1]);
        atomicAdd(&a.g_means[3 * (long long)g + 2], gxs[2]);
      }
    }
  }
}

template <int H, int L>
cudaError_t launch_mlp_tile(const MlpBwdArgs& a, cudaStream_t s) {
  constexpr int HL = H * L;
  const size_t smem = sizeof(float) * ((size_t)a.f.mg.total + (size_t)(HL + 5 * kWidth + kDeltaDim) * kTS) +
                      kTG * sizeof(float4) + kTG * sizeof(int);
  static PerDeviceFlag attr;
  cudaError_t e = once_per_device(attr, [&] {
    return cudaFuncSetAttribute(mlp_bwd_tile_kernel<H, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
  const int sms = device_sm_count();
  const long long need = ((long long)a.f.n + kTG - 1) / kTG;
  const int grid = (int)(need < sms ? need : sms);
  mlp_bwd_tile_kernel<H, L><<<grid, kTT, smem, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ weight gradients

constexpr int kWChunk = 256;   // Gaussians per partial (~400 chunks per layer at 100k Gaussians)
constexpr int kWStage = 32;    // Gaussians staged per step
constexpr int kWBlocks = 2;    // 4x4 output blocks per thread (a 96-input layer has 16 x 24 = 384)

// Partial sums over one chunk of Gaussians of dW[o][i] = sum_n D[o][n] X[i][n] and
// db[o] = sum_n D[o][n], register-blocked: the (O/4) x (I/4) blocks of 4x4 weights
// are spread over the threads, each reading 4 D and 4 X values (two 128-bit shared
// loads) per staged Gaussian for 16 FMAs; the threads of the first column block
// also sum the bias.  A layer with fewer blocks than threads (the 3- and 4-output
// head layers) splits the staged Gaussians among threads and adds the slices up
// in shared memory at the end.
__global__ void __launch_bounds__(256) wgrad_partial_kernel(const __grid_constant__ WgradArgs wa) {
  const WgradLayer& ly = wa.l[blockIdx.y];
  const float* __restrict__ D = ly.D;
  const float* __restrict__ X = ly.X;
  const long long n = wa.n;
  const int O = ly.O, I = ly.I;
  float* __restrict__ partial = wa.partial + ly.part_off;
  // two stages of D [kWStage][64] and X [kWStage][96] (the next one loading by
  // cp.async while this one is multiplied); rows padded to 68 and 100 floats, so that
  // a warp's transposing stores (one Gaussian per lane) spread over 8 banks, not 1;
  // after the loop the same memory holds the slices' sums
  constexpr int kDS = 68, kXS = 100;
  __shared__ __align__(16) float sBuf[2 * kWStage * kDS + 2 * kWStage * kXS];
  float (*sD)[kWStage][kDS] = reinterpret_cast<float (*)[kWStage][kDS]>(sBuf);
  float (*sX)[kWStage][kXS] = reinterpret_cast<float (*)[kWStage][kXS]>(sBuf + 2 * kWStage * kDS);
  float (*sRed)[20] = reinterpret_cast<float (*)[20]>(sBuf);
  static_assert(256 * 20 <= 2 * kWStage * kDS + 2 * kWStage * kXS, "slice sums fit in the stage buffers");
  const int E = O * I + O;
  const int IB = I / 4, OB = (O + 3) / 4, NB = OB * IB;
  const int ks = NB >= 256 ? 1 : 256 / NB;  // slices of the staged Gaussians
  const int slice = threadIdx.x / (NB < 256 ? NB : 256);
  const long long n0 = (long long)blockIdx.x * kWChunk;
  const long long n1 = min(n, n0 + kWChunk);
  float acc[kWBlocks][16], bacc[kWBlocks][4];
#pragma unroll
  for (int b = 0; b < kWBlocks; ++b) {
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[b][k] = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) bacc[b][k] = 0.f;
  }
  // one stage into buffer `buf`: 4-byte copies (the arrays are transposed on the way)
  auto stage = [&](int buf, long long b0) {
    const int m = (int)min((long long)kWStage, n1 - b0);
    for (int t = threadIdx.x; t < kWStage * 64; t += 256) {
      const int o = t / kWStage, j = t % kWStage;
      float* dst = &sD[buf][j][o];
      if (j < m && o < O) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                     "l"(D + (long long)o * n + b0 + j)
                     : "memory");
      } else {
        *dst = 0.f;
      }
    }
    for (int t = threadIdx.x; t < kWStage * I; t += 256) {
      const int i = t / kWStage, j = t % kWStage;
      float* dst = &sX[buf][j][i];
      if (j < m) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                     "l"(X + (long long)i * n + b0 + j)
                     : "memory");
      } else {
        *dst = 0.f;
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  if (n0 < n1) stage(0, n0);
  int buf = 0;
  for (long long b0 = n0; b0 < n1; b0 += kWStage, buf ^= 1) {
    // the next stage into the other buffer (last read by the previous step, before its
    // closing barrier), then wait for this one
    if (b0 + kWStage < n1) {
      stage(buf ^ 1, b0 + kWStage);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    if (slice < ks) {
#pragma unroll
      for (int b = 0; b < kWBlocks; ++b) {
        const int blk = (NB < 256 ? threadIdx.x % NB : threadIdx.x) + 256 * b;
        if (blk >= NB || (b > 0 && NB < 256)) break;
        const int ob = blk / IB, ib = blk % IB;
        float* a = acc[b];
#pragma unroll 4
        for (int j = slice; j < kWStage; j += ks) {
          const float4 d4 = *reinterpret_cast<const float4*>(&sD[buf][j][4 * ob]);
          const float4 x4 = *reinterpret_cast<const float4*>(&sX[buf][j][4 * ib]);
          const float dv[4] = {d4.x, d4.y, d4.z, d4.w};
          const float2 x01 = make_float2(x4.x, x4.y), x23 = make_float2(x4.z, x4.w);
#pragma unroll
          for (int r = 0; r < 4; ++r) {  // column pairs: one f32x2 FMA per two (the same FP32 FMAs)
            const float2 dr = make_float2(dv[r], dv[r]);
            float2 p0 = make_float2(a[4 * r], a[4 * r + 1]), p1 = make_float2(a[4 * r + 2], a[4 * r + 3]);
            p0 = __ffma2_rn(dr, x01, p0);
            p1 = __ffma2_rn(dr, x23, p1);
            a[4 * r] = p0.x; a[4 * r + 1] = p0.y; a[4 * r + 2] = p1.x; a[4 * r + 3] = p1.y;
          }
          if (ib == 0)
#pragma unroll
            for (int r = 0; r < 4; ++r) bacc[b][r] += dv[r];
        }
      }
    }
    __syncthreads();  // this buffer is refilled two steps on
  }
  if (ks > 1) {  // add the slices up: slice 0 of each block collects the others
    __syncthreads();
    if (slice < ks) {
      for (int k = 0; k < 16; ++k) sRed[threadIdx.x][k] = acc[0][k];
      for (int k = 0; k < 4; ++k) sRed[threadIdx.x][16 + k] = bacc[0][k];
    }
    __syncthreads();
    if (slice == 0) {
      for (int sl = 1; sl < ks; ++sl) {
        const int src = threadIdx.x + sl * NB;
        for (int k = 0; k < 16; ++k) acc[0][k] += sRed[src][k];
        for (int k = 0; k < 4; ++k) bacc[0][k] += sRed[src][16 + k];
      }
    }
  }
  if (slice != 0) return;
  // entry layout: W[o][i] at o * I + i, then b[o] at O * I + o
#pragma unroll
  for (int b = 0; b < kWBlocks; ++b) {
    const int blk = (NB < 256 ? threadIdx.x % NB : threadIdx.x) + 256 * b;
    if (blk >= NB || (b > 0 && NB < 256)) break;
    const int ob = blk / IB, ib = blk % IB;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int o = 4 * ob + r;
      if (o >= O) continue;
#pragma unroll
      for (int c = 0; c < 4; ++c) partial[(long long)blockIdx.x * E + o * I + 4 * ib + c] = acc[b][4 * r + c];
      if (ib == 0) partial[(long long)blockIdx.x * E + O * I + o] = bacc[b][r];
    }
  }
}

// Four threads per weight (adjacent lanes), each summing every fourth chunk in
// eight running sums (eight loads in flight), then the four combined by two
// shuffles: a fixed order, so the result is deterministic.
constexpr int kRedSplit = 4;
__global__ void wgrad_reduce_kernel(const __grid_constant__ WgradArgs wa) {
  const WgradLayer& ly = wa.l[blockIdx.y];
  const int O = ly.O, I = ly.I;
  const int E = O * I + O;
  const int e = blockIdx.x * (blockDim.x / kRedSplit) + (int)threadIdx.x / kRedSplit;
  const int split = (int)threadIdx.x % kRedSplit;
  const bool live = e < E;  // (every lane stays for the shuffles)
  const float* partial = wa.partial + ly.part_off;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (live) {
    int c = split, k = 0;
    for (; c + 7 * kRedSplit < wa.chunks; c += 8 * kRedSplit) {
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] += partial[(long long)(c + u * kRedSplit) * E + e];
    }
    for (; c < wa.chunks; c += kRedSplit, ++k) acc[k & 7] += partial[(long long)c * E + e];
  }
  float s = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  if (!live || split != 0) return;
  if (e < O * I)
    ly.gW[e] += s;
  else
    ly.gb[e - O * I] += s;
}

}  // namespace

cudaError_t launch_composite_bwd(const CompositeBwdArgs& a, cudaStream_t s) {
  const int tiles_y = (a.height + kTile - 1) / kTile;
  if (a.tiles_x * tiles_y == 0) return cudaSuccess;
  composite_bwd_kernel<<<a.tiles_x * tiles_y, kBatch, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_project_bwd(const ProjectBwdArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  project_bwd_kernel<<<(a.n + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mlp_bwd(const MlpBwdArgs& a, cudaStream_t s) {
  if (a.f.n <= 0) return cudaSuccess;
  const int h = a.f.pg.feat_dim, L = a.f.pg.n_levels;
  if (h == 16 && L == 1) return launch_mlp_tile<16, 1>(a, s);
  if (h == 16 && L == 2) return launch_mlp_tile<16, 2>(a, s);
  if (h == 16 && L == 3) return launch_mlp_tile<16, 3>(a, s);
  if (h == 32 && L == 1) return launch_mlp_tile<32, 1>(a, s);
  if (h == 32 && L == 2) return launch_mlp_tile<32, 2>(a, s);
  if (h == 32 && L == 3) return launch_mlp_tile<32, 3>(a, s);
  return cudaErrorInvalidValue;
}

long long wgrad_chunks(long long n) { return (n + kWChunk - 1) / kWChunk; }

cudaError_t launch_wgrad(WgradArgs& a, cudaStream_t s) {
  if (a.n <= 0 || a.n_layers <= 0) return cudaSuccess;
  a.chunks = (int)wgrad_chunks(a.n);
  int maxE = 0;
  long long off = 0;
  for (int k = 0; k < a.n_layers; ++k) {
    if (a.l[k].O > 64 || a.l[k].I > 96 || (a.l[k].I & 3)) return cudaErrorInvalidValue;
    const int E = a.l[k].O * a.l[k].I + a.l[k].O;
    a.l[k].part_off = off;
    off += (long long)a.chunks * E;
    maxE = std::max(maxE, E);
  }
  wgrad_partial_kernel<<<dim3(a.chunks, a.n_layers), 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  wgrad_reduce_kernel<<<dim3((maxE + 256 / kRedSplit - 1) / (256 / kRedSplit), a.n_layers), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fs4d
