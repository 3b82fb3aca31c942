// Gaussian deformation field, float32 SIMT path (Sec. 4.2, Eq. 5, Eq. 6).
//
// One thread per (timestamp, Gaussian).  Per thread:
//   1. normalise (x, y, z) by the scene box and t to [-1, 1];
//   2. for every level, bilinearly interpolate the six planes xy xz yz xt yt zt
//      (channels-last, so each grid vertex is h contiguous floats read as 128-bit
//      vectors through the read-only path) and multiply them channel-wise (Eq. 5);
//   3. run phi_d (two ReLU layers) and the heads phi_x, phi_r, phi_s;
//   4. add the deltas to X, r, s (Eq. 6).
// The CTA keeps every MLP layer transposed (Wt[in][out]) in shared memory, so a
// single broadcast 128-bit load feeds four accumulators.  Activations live in a
// per-thread column of a shared [rows][threads] array (conflict-free), which
// lets the input loop stay rolled while 64 accumulators stay in registers.
// The grid is persistent: one CTA per SM, weights copied once per CTA.
#include "fs4d_internal.cuh"

namespace fs4d {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void axis_setup(float u, int R, int& i0, float& f) {
  const float uc = fminf(1.f, fmaxf(-1.f, u));
  const float g = (uc + 1.f) * 0.5f * (float)(R - 1);
  int i = (int)floorf(g);
  i = max(0, min(i, R - 2));
  i0 = i;
  f = g - (float)i;
}

template <int IN>
__device__ __forceinline__ void dense64(const float* __restrict__ Wt, const float* __restrict__ b,
                                        const float* __restrict__ col, float (&y)[kWidth]) {
#pragma unroll
  for (int o = 0; o < kWidth; ++o) y[o] = b[o];
#pragma unroll 2
  for (int i = 0; i < IN; ++i) {
    const float x = col[i * kThreads];
    const float4* w = reinterpret_cast<const float4*>(Wt + i * kWidth);
#pragma unroll
    for (int q = 0; q < kWidth / 4; ++q) {
      const float4 ww = w[q];
      y[4 * q + 0] = fmaf(ww.x, x, y[4 * q + 0]);
      y[4 * q + 1] = fmaf(ww.y, x, y[4 * q + 1]);
      y[4 * q + 2] = fmaf(ww.z, x, y[4 * q + 2]);
      y[4 * q + 3] = fmaf(ww.w, x, y[4 * q + 3]);
    }
  }
}

// One head: out = W2 relu(W1 f_d + b1) + b2, W2 stored transposed [64][OUT].
template <int OUT>
__device__ __forceinline__ void head(const float* __restrict__ sw, const MlpGeomT& mg, int layer,
                                     const float* __restrict__ col, float* out) {
  float y[kWidth];
  dense64<kWidth>(sw + mg.w[layer], sw + mg.b[layer], col, y);
  const float* W2 = sw + mg.w[layer + 1];
  const float* b2 = sw + mg.b[layer + 1];
#pragma unroll
  for (int j = 0; j < OUT; ++j) out[j] = b2[j];
#pragma unroll
  for (int o = 0; o < kWidth; ++o) {
    const float h = fmaxf(y[o], 0.f);
#pragma unroll
    for (int j = 0; j < OUT; ++j) out[j] = fmaf(W2[o * OUT + j], h, out[j]);
  }
}

template <int H, int L>
__global__ void __launch_bounds__(kThreads, 1) deform_fp32_kernel(DeformArgs a) {
  constexpr int HL = H * L;
  extern __shared__ float4 smem4[];
  float* sw = reinterpret_cast<float*>(smem4);
  float* act = sw + a.mg.total;
  for (int i = threadIdx.x; i < a.mg.total / 4; i += kThreads)
    smem4[i] = __ldg(reinterpret_cast<const float4*>(a.mlp_t) + i);
  __syncthreads();

  const PlaneGeom& pg = a.pg;
  float* col = act + threadIdx.x;
  const long long total = (long long)a.n * a.n_t;
  for (long long gi = (long long)blockIdx.x * kThreads + threadIdx.x; gi < total;
       gi += (long long)gridDim.x * kThreads) {
    const int ti = (int)(gi / a.n);
    const int gw = (int)(gi - (long long)ti * a.n);
    const int g = a.perm ? (int)a.perm[gw] : gw;  // spatially coherent work order
    const float t = a.ts ? a.ts[ti] : a.t0;
    const float X0 = a.means[3 * g], X1 = a.means[3 * g + 1], X2 = a.means[3 * g + 2];
    float c[4];
    c[0] = (X0 - pg.aabb_min[0]) * pg.aabb_scale[0] - 1.f;
    c[1] = (X1 - pg.aabb_min[1]) * pg.aabb_scale[1] - 1.f;
    c[2] = (X2 - pg.aabb_min[2]) * pg.aabb_scale[2] - 1.f;
    c[3] = 2.f * t - 1.f;

    // Eq. 5: f_h = concat_l prod_p interp(R_l,p)
#pragma unroll
    for (int l = 0; l < L; ++l) {
      float f[H];
#pragma unroll
      for (int k = 0; k < H; ++k) f[k] = 1.f;
#pragma unroll
      for (int p = 0; p < 6; ++p) {
        const int ax = (p < 2) ? 0 : (p == 2 ? 1 : p - 3);  // xy xz yz xt yt zt
        const int bx = (p == 0) ? 1 : (p <= 2 ? 2 : 3);
        const int Ra = ax < 3 ? pg.res[l] : pg.res_time;
        const int Rb = bx < 3 ? pg.res[l] : pg.res_time;
        int i0, j0;
        float fa, fb;
        axis_setup(c[ax], Ra, i0, fa);
        axis_setup(c[bx], Rb, j0, fb);
        const float4* v00 = reinterpret_cast<const float4*>(a.planes + pg.off[l][p] + ((long long)j0 * Ra + i0) * H);
        const float4* v10 = v00 + H / 4;
        const float4* v01 = v00 + (long long)Ra * (H / 4);
        const float4* v11 = v01 + H / 4;
        const float w00 = (1.f - fa) * (1.f - fb), w10 = fa * (1.f - fb), w01 = (1.f - fa) * fb, w11 = fa * fb;
#pragma unroll
        for (int q = 0; q < H / 4; ++q) {
          const float4 A = __ldg(v00 + q), B = __ldg(v10 + q), C = __ldg(v01 + q), D = __ldg(v11 + q);
          f[4 * q + 0] *= w00 * A.x + w10 * B.x + w01 * C.x + w11 * D.x;
          f[4 * q + 1] *= w00 * A.y + w10 * B.y + w01 * C.y + w11 * D.y;
          f[4 * q + 2] *= w00 * A.z + w10 * B.z + w01 * C.z + w11 * D.z;
          f[4 * q + 3] *= w00 * A.w + w10 * B.w + w01 * C.w + w11 * D.w;
        }
      }
#pragma unroll
      for (int k = 0; k < H; ++k) col[(l * H + k) * kThreads] = f[k];
    }

    // phi_d: two ReLU layers; f_d ends in rows 0..63 of the column.
    float y[kWidth];
    dense64<HL>(sw + a.mg.w[0], sw + a.mg.b[0], col, y);
#pragma unroll
    for (int o = 0; o < kWidth; ++o) col[o * kThreads] = fmaxf(y[o], 0.f);
    dense64<kWidth>(sw + a.mg.w[1], sw + a.mg.b[1], col, y);
#pragma unroll
    for (int o = 0; o < kWidth; ++o) col[o * kThreads] = fmaxf(y[o], 0.f);

    // Heads phi_x, phi_r, phi_s and Eq. 6.
    float d[kDeltaDim];
    head<3>(sw, a.mg, 2, col, d);
    head<4>(sw, a.mg, 4, col, d + 3);
    head<3>(sw, a.mg, 6, col, d + 7);
    const long long o = a.out_tab ? g : (long long)ti * a.n + g;
    float* om = a.out_tab ? a.out_tab[3 * ti] : a.out_means;
    float* oq = a.out_tab ? a.out_tab[3 * ti + 1] : a.out_quats;
    float* os = a.out_tab ? a.out_tab[3 * ti + 2] : a.out_log_scales;
    om[3 * o + 0] = X0 + d[0];
    om[3 * o + 1] = X1 + d[1];
    om[3 * o + 2] = X2 + d[2];
    const float4 q = reinterpret_cast<const float4*>(a.quats)[g];
    reinterpret_cast<float4*>(oq)[o] = make_float4(q.x + d[3], q.y + d[4], q.z + d[5], q.w + d[6]);
    os[3 * o + 0] = a.log_scales[3 * g + 0] + d[7];
    os[3 * o + 1] = a.log_scales[3 * g + 1] + d[8];
    os[3 * o + 2] = a.log_scales[3 * g + 2] + d[9];
  }
}

template <int H, int L>
cudaError_t launch_t(const DeformArgs& a, cudaStream_t s) {
  constexpr int HL = H * L;
  constexpr int rows = HL > kWidth ? HL : kWidth;
  const size_t smem = sizeof(float) * ((size_t)a.mg.total + (size_t)rows * kThreads);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(deform_fp32_kernel<H, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const long long total = (long long)a.n * a.n_t;
  const long long need = (total + kThreads - 1) / kThreads;
  const int grid = (int)(need < sms ? need : sms);
  deform_fp32_kernel<H, L><<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool deform_fp32_supported(int feat_dim, int n_levels) {
  return (feat_dim == 16 || feat_dim == 32) && n_levels >= 1 && n_levels <= 3;
}

cudaError_t launch_deform_fp32(const DeformArgs& a, cudaStream_t s) {
  if ((long long)a.n * a.n_t == 0) return cudaSuccess;
  const int h = a.pg.feat_dim, L = a.pg.n_levels;
  if (h == 16 && L == 1) return launch_t<16, 1>(a, s);
  if (h == 16 && L == 2) return launch_t<16, 2>(a, s);
  if (h == 16 && L == 3) return launch_t<16, 3>(a, s);
  if (h == 32 && L == 1) return launch_t<32, 1>(a, s);
  if (h == 32 && L == 2) return launch_t<32, 2>(a, s);
  if (h == 32 && L == 3) return launch_t<32, 3>(a, s);
  return cudaErrorInvalidValue;
}

}  // namespace fs4d
