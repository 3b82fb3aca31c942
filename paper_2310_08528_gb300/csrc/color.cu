// Colour and opacity deformation (App. B), float32 path: two more heads on the
// deformation feature f_d, each Lin(64 -> 64), ReLU, Lin(64 -> out) like phi_x,
// phi_r, phi_s:
//   C' = C + phi_C(f_d)            (every SH coefficient, out = 3K)
//   logit' = logit + phi_alpha(f_d) (the opacity as stored, out = 1)
// The FP32 deformation kernel leaves f_d (after phi_d's second ReLU) in work
// order.  Persistent CTAs of 256 threads take tiles of 128 Gaussians: f_d is
// transposed into shared memory (feature-major) and each layer is a register-
// blocked SIMT GEMM -- a thread computes 4 Gaussians x 8 outputs with f32x2 FMAs
// on output pairs, every output summed from its bias in input order, the same
// float32 arithmetic per element as one thread per Gaussian -- over weights held
// transposed in shared memory.  It writes the frame's deformed SH and opacity
// logits, which the projection then reads in place of the scene's.
#include "fs4d_internal.cuh"

namespace fs4d {
namespace {

constexpr int kThreads = 256;
constexpr int kW = 64;
constexpr int kTileG = 128;      // Gaussians per tile
constexpr int kGS = kTileG + 4;  // row stride (floats) of the activation arrays
constexpr int kOutC = 48;        // colour outputs, padded with zero weights (3K <= 48)

// Shared memory (floats): the weights transposed, Wt[in][out], and the biases of
// c1 c2 a1 a2, then the activations F [64][kGS] (f_d) and H [64][kGS] (the hidden
// layer of the head being evaluated).  Every row start is 16-byte aligned.
constexpr int kC1 = 0;
constexpr int kC1b = kC1 + kW * kW;
constexpr int kC2 = kC1b + kW;
constexpr int kC2b = kC2 + kW * kOutC;
constexpr int kA1 = kC2b + kOutC;
constexpr int kA1b = kA1 + kW * kW;
constexpr int kA2 = kA1b + kW;
constexpr int kA2b = kA2 + kW;
constexpr int kF = (kA2b + 1 + 3) & ~3;
constexpr int kH = kF + kW * kGS;
constexpr int kTotal = kH + kW * kGS;

// acc[g][o] = b[o8 + o] + sum_i Wt[i][o8 + o] src[i][g4 + g], in input order, for
// the thread's 4 Gaussians (g4..) and 8 outputs (o8..) of a 64-input layer.
__device__ __forceinline__ void tile_layer(const float* __restrict__ Wt, int ldo, const float* __restrict__ b,
                                           const float* __restrict__ src, int g4, int o8, float (&acc)[4][8]) {
  float2 a2[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const float2 bp = make_float2(b[o8 + 2 * p], b[o8 + 2 * p + 1]);
#pragma unroll
    for (int g = 0; g < 4; ++g) a2[g][p] = bp;
  }
#pragma unroll 4
  for (int i = 0; i < kW; ++i) {
    const float4 x = *reinterpret_cast<const float4*>(src + i * kGS + g4);
    const float4 w0 = *reinterpret_cast<const float4*>(Wt + i * ldo + o8);
    const float4 w1 = *reinterpret_cast<const float4*>(Wt + i * ldo + o8 + 4);
    const float xs[4] = {x.x, x.y, x.z, x.w};
    const float2 ws[4] = {make_float2(w0.x, w0.y), make_float2(w0.z, w0.w), make_float2(w1.x, w1.y),
                          make_float2(w1.z, w1.w)};
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const float2 xg = make_float2(xs[g], xs[g]);
#pragma unroll
      for (int p = 0; p < 4; ++p) a2[g][p] = __ffma2_rn(ws[p], xg, a2[g][p]);
    }
  }
#pragma unroll
  for (int g = 0; g < 4; ++g)
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      acc[g][2 * p] = a2[g][p].x;
      acc[g][2 * p + 1] = a2[g][p].y;
    }
}

// dst[o8 + o][g4 + g] = relu(acc[g][o])
__device__ __forceinline__ void store_relu(float* __restrict__ dst, int g4, int o8, const float (&acc)[4][8]) {
#pragma unroll
  for (int o = 0; o < 8; ++o)
    *reinterpret_cast<float4*>(dst + (o8 + o) * kGS + g4) =
        make_float4(fmaxf(acc[0][o], 0.f), fmaxf(acc[1][o], 0.f), fmaxf(acc[2][o], 0.f), fmaxf(acc[3][o], 0.f));
}

__global__ void __launch_bounds__(kThreads, 2) color_heads_kernel(const ColorArgs a) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const int tid = threadIdx.x;
  const int k3 = a.k3;
  // the source layout: W_C1 [64][64], b_C1, W_C2 [3K][64], b_C2, W_a1, b_a1, W_a2 [64], b_a2
  const float* w = a.weights;
  const int c1w = 0, c1b = kW * kW, c2w = c1b + kW, c2b = c2w + k3 * kW, a1w = c2b + k3, a1b = a1w + kW * kW,
            a2w = a1b + kW, a2b = a2w + kW;
  for (int e = tid; e < kW * kW; e += kThreads) {  // e = o * 64 + i  ->  Wt[i][o]
    const int o = e / kW, i = e % kW;
    sm[kC1 + i * kW + o] = w[c1w + e];
    sm[kA1 + i * kW + o] = w[a1w + e];
  }
  for (int e = tid; e < kOutC * kW; e += kThreads) {
    const int o = e / kW, i = e % kW;
    sm[kC2 + i * kOutC + o] = o < k3 ? w[c2w + o * kW + i] : 0.f;
  }
  for (int e = tid; e < kW; e += kThreads) {
    sm[kC1b + e] = w[c1b + e];
    sm[kA1b + e] = w[a1b + e];
    sm[kA2 + e] = w[a2w + e];
  }
  for (int e = tid; e < kOutC; e += kThreads) sm[kC2b + e] = e < k3 ? w[c2b + e] : 0.f;
  if (tid == 0) sm[kA2b] = w[a2b];
  const int lane = tid & 31, warp = tid >> 5;
  const int g4 = lane * 4, o8 = warp * 8;
  const long long tiles = ((long long)a.n + kTileG - 1) / kTileG;
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long long base = tile * kTileG;
    __syncthreads();  // the weights are in; the previous tile is done with F and H
    // f_d rows -> F [feature][Gaussian]
    for (int e = tid; e < kTileG * (kW / 4); e += kThreads) {
      const int r = e / (kW / 4), k4 = (e % (kW / 4)) * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (base + r < a.n) v = __ldg(reinterpret_cast<const float4*>(a.fd + (size_t)(base + r) * kW + k4));
      sm[kF + (k4 + 0) * kGS + r] = v.x;
      sm[kF + (k4 + 1) * kGS + r] = v.y;
      sm[kF + (k4 + 2) * kGS + r] = v.z;
      sm[kF + (k4 + 3) * kGS + r] = v.w;
    }
    __syncthreads();
    float acc[4][8];
    // ---- phi_C: hidden layer into H, then the 3K outputs added to the SH
    tile_layer(sm + kC1, kW, sm + kC1b, sm + kF, g4, o8, acc);
    store_relu(sm + kH, g4, o8, acc);
    __syncthreads();
    if (o8 < k3) {  // warp-uniform: the warps whose outputs hold colour coefficients
      tile_layer(sm + kC2, kOutC, sm + kC2b, sm + kH, g4, o8, acc);
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const long long gi = base + g4 + g;
        if (gi >= a.n) continue;
        const size_t gg = a.perm ? (size_t)a.perm[gi] : (size_t)gi;
#pragma unroll
        for (int o = 0; o < 8; ++o)
          if (o8 + o < k3) a.sh_out[gg * k3 + o8 + o] = a.sh[gg * k3 + o8 + o] + acc[g][o];
      }
    }
    __syncthreads();  // H is rewritten below
    // ---- phi_alpha: hidden layer into H, then one output per Gaussian
    tile_layer(sm + kA1, kW, sm + kA1b, sm + kF, g4, o8, acc);
    store_relu(sm + kH, g4, o8, acc);
    __syncthreads();
    if (tid < kTileG && base + tid < a.n) {
      float s = sm[kA2b];
#pragma unroll 8
      for (int o = 0; o < kW; ++o) s = fmaf(sm[kA2 + o], sm[kH + o * kGS + tid], s);
      const size_t gg = a.perm ? (size_t)a.perm[base + tid] : (size_t)(base + tid);
      a.logit_out[gg] = a.logits[gg] + s;
    }
  }
}

}  // namespace

int color_layer_floats(int k3) { return 2 * (kW * kW + kW) + k3 * kW + k3 + kW + 1; }

cudaError_t launch_color_heads(const ColorArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (a.k3 < 3 || a.k3 > kOutC || (reinterpret_cast<uintptr_t>(a.fd) & 15u)) return cudaErrorInvalidValue;
  const size_t smem = 4 * (size_t)kTotal;
  static PerDeviceFlag attr;
  cudaError_t e = once_per_device(attr, [&] {
    return cudaFuncSetAttribute(color_heads_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
  const long long tiles = ((long long)a.n + kTileG - 1) / kTileG;
  const int sms = device_sm_count();
  const int grid = (int)(tiles < 2LL * sms ? tiles : 2LL * sms);
  color_heads_kernel<<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fs4d
