// Colour and opacity deformation (App. B): two more heads on the deformation
// feature f_d, each Lin(64 -> 64), ReLU, Lin(64 -> out) like phi_x, phi_r, phi_s:
//   C' = C + phi_C(f_d)            (every SH coefficient, out = 3K)
//   logit' = logit + phi_alpha(f_d) (the opacity as stored, out = 1)
// The deformation kernels leave f_d (float32, after phi_d's second ReLU) in work
// order; one thread per Gaussian runs both heads in float32 with the weights in
// shared memory (read as broadcasts) and writes the frame's deformed SH and
// opacity logits, which the projection then reads in place of the scene's.
// FMA-bound SIMT work (~11.4k FMA per Gaussian), off the path of scenes without
// these heads.
#include "fs4d_internal.cuh"

namespace fs4d {
namespace {

constexpr int kThreads = 128;
constexpr int kW = 64;

// Shared-memory layout of the four layers (each weight block 16-byte aligned):
// c1 W [64][64], c1 b [64], c2 W [3K][64], c2 b [3K], a1 W, a1 b, a2 W [64], a2 b.
struct ColorSmem {
  int c1w, c1b, c2w, c2b, a1w, a1b, a2w, a2b, total;
};
__host__ __device__ inline ColorSmem color_smem(int k3) {
  ColorSmem m;
  m.c1w = 0;
  m.c1b = kW * kW;
  m.c2w = m.c1b + kW;
  m.c2b = m.c2w + k3 * kW;
  m.a1w = (m.c2b + k3 + 3) & ~3;
  m.a1b = m.a1w + kW * kW;
  m.a2w = m.a1b + kW;
  m.a2b = m.a2w + kW;
  m.total = m.a2b + 1;
  return m;
}

// y[o] = relu(b[o] + sum_i W[o][i] x[i]) for a 64 x 64 layer.
__device__ __forceinline__ void hidden64(const float* __restrict__ w, const float* __restrict__ b,
                                         const float (&x)[kW], float (&y)[kW]) {
#pragma unroll
  for (int o = 0; o < kW; ++o) {
    const float4* row = reinterpret_cast<const float4*>(w + o * kW);
    float acc = b[o];
#pragma unroll
    for (int i = 0; i < kW / 4; ++i) {
      const float4 v = row[i];
      acc = fmaf(v.x, x[4 * i], acc);
      acc = fmaf(v.y, x[4 * i + 1], acc);
      acc = fmaf(v.z, x[4 * i + 2], acc);
      acc = fmaf(v.w, x[4 * i + 3], acc);
    }
    y[o] = fmaxf(acc, 0.f);
  }
}

// bias + sum_i row[i] h[i] for one output of a layer (row: 64 weights, 16-byte aligned).
__device__ __forceinline__ float out_row(const float* __restrict__ row_w, float bias, const float (&h)[kW]) {
  const float4* row = reinterpret_cast<const float4*>(row_w);
  float acc = bias;
#pragma unroll
  for (int i = 0; i < kW / 4; ++i) {
    const float4 v = row[i];
    acc = fmaf(v.x, h[4 * i], acc);
    acc = fmaf(v.y, h[4 * i + 1], acc);
    acc = fmaf(v.z, h[4 * i + 2], acc);
    acc = fmaf(v.w, h[4 * i + 3], acc);
  }
  return acc;
}

__global__ void __launch_bounds__(kThreads) color_heads_kernel(const ColorArgs a) {
  extern __shared__ float4 smem4[];
  float* sw = reinterpret_cast<float*>(smem4);
  const ColorSmem m = color_smem(a.k3);
  // the source layout is contiguous (W then b per layer); a1 may move up to 3 floats
  const int src_a1 = m.c2b + a.k3;
  for (int i = threadIdx.x; i < src_a1; i += kThreads) sw[i] = a.weights[i];
  for (int i = threadIdx.x; i < m.total - m.a1w; i += kThreads) sw[m.a1w + i] = a.weights[src_a1 + i];
  __syncthreads();
  const int i = blockIdx.x * kThreads + threadIdx.x;
  if (i >= a.n) return;
  const int g = a.perm ? (int)a.perm[i] : i;
  float f[kW];
  const float4* src = reinterpret_cast<const float4*>(a.fd + (size_t)i * kW);
#pragma unroll
  for (int k = 0; k < kW / 4; ++k) {
    const float4 v = src[k];
    f[4 * k] = v.x;
    f[4 * k + 1] = v.y;
    f[4 * k + 2] = v.z;
    f[4 * k + 3] = v.w;
  }
  float h[kW];
  hidden64(sw + m.c1w, sw + m.c1b, f, h);
  const float* sh = a.sh + (size_t)g * a.k3;
  float* sh_out = a.sh_out + (size_t)g * a.k3;
  for (int o = 0; o < a.k3; ++o) sh_out[o] = sh[o] + out_row(sw + m.c2w + o * kW, sw[m.c2b + o], h);
  hidden64(sw + m.a1w, sw + m.a1b, f, h);
  a.logit_out[g] = a.logits[g] + out_row(sw + m.a2w, sw[m.a2b], h);
}

}  // namespace

int color_layer_floats(int k3) { return 2 * (kW * kW + kW) + k3 * kW + k3 + kW + 1; }

cudaError_t launch_color_heads(const ColorArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (a.k3 < 3 || a.k3 > 48 || (reinterpret_cast<uintptr_t>(a.fd) & 15u)) return cudaErrorInvalidValue;
  const size_t smem = 4 * (size_t)color_smem(a.k3).total;
  static PerDeviceFlag attr;
  cudaError_t e = once_per_device(attr, [&] {
    return cudaFuncSetAttribute(color_heads_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                4 * color_smem(48).total);
  });
  if (e != cudaSuccess) return e;
  color_heads_kernel<<<(a.n + kThreads - 1) / kThreads, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fs4d
