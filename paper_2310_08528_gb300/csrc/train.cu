// Training step kernels (Sec. 4.3, App. A): the L1 colour loss and its gradient,
// the grid total-variation loss over the HexPlane and its gradient, one Adam
// update of every parameter group, and the refresh of the derived device copies
// (BF16 planes, transposed MLP, tensor-core operand image) from the updated
// float32 parameters.  Every kernel is a single streaming pass over its arrays
// (HBM-bound): coalesced loads, grid-stride loops over a grid sized from the
// device's SM count, deterministic two-stage loss reductions.
#include <algorithm>

#include "fs4d_internal.cuh"

namespace fs4d {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float block_sum(float v, float* tmp) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) tmp[warp] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x == 0)
    for (int w = 0; w < kThreads / 32; ++w) s += tmp[w];
  __syncthreads();
  return s;  // valid in thread 0
}

// |I^ - I| summed per block; dL/dI = sign(I^ - I) / count (0 where equal).
// n4: float4 groups taken by 128-bit accesses (0 when a pointer is not 16-byte aligned).
__global__ void __launch_bounds__(kThreads) l1_kernel(const float* __restrict__ img, const float* __restrict__ tgt,
                                                      long long count, long long n4, float inv_count,
                                                      float* __restrict__ dl, float* __restrict__ partial) {
  __shared__ float tmp[kThreads / 32];
  float acc = 0.f;
  const float4* a4 = reinterpret_cast<const float4*>(img);
  const float4* b4 = reinterpret_cast<const float4*>(tgt);
  float4* d4 = reinterpret_cast<float4*>(dl);
  auto sg = [inv_count](float d) { return d > 0.f ? inv_count : (d < 0.f ? -inv_count : 0.f); };
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n4; i += (long long)gridDim.x * kThreads) {
    const float4 a = a4[i], b = b4[i];
    const float4 d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
    acc += (fabsf(d.x) + fabsf(d.y)) + (fabsf(d.z) + fabsf(d.w));
    d4[i] = make_float4(sg(d.x), sg(d.y), sg(d.z), sg(d.w));
  }
  for (long long i = 4 * n4 + blockIdx.x * (long long)kThreads + threadIdx.x; i < count;
       i += (long long)gridDim.x * kThreads) {
    const float d = img[i] - tgt[i];
    acc += fabsf(d);
    dl[i] = sg(d);
  }
  const float s = block_sum(acc, tmp);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out = scale * (sum of the partials), in double, by one block in a fixed order.
__global__ void __launch_bounds__(kThreads) finish_sum_kernel(const float* __restrict__ partial, int n, double scale,
                                                              float* __restrict__ out) {
  __shared__ double tmp[kThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kThreads) s += (double)partial[i];
  tmp[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) tmp[threadIdx.x] += tmp[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = (float)(scale * tmp[0]);
}

// One plane of the HexPlane, as the TV kernel sees it.
struct TvPlane {
  long long off;   // element offset of [R_b][R_a][h]
  long long cells; // R_b * R_a * h
  int ra, rb;
  float wa, wb;    // 2 weight / n_a, 2 weight / n_b (gradient factors); n_* = neighbour pairs x h
};
struct TvArgs {
  TvPlane p[24];
  int n_planes;
  int h;
  long long total;
};

// Grid TV (reading of L_tv): per plane, mean squared neighbour difference along each
// axis.  Each element's gradient needs only its 4 neighbours, so every element is
// written by exactly one thread (g += ...), no atomics.  Per-block partial of the
// loss (each pair counted by the element on its lower side).
__global__ void __launch_bounds__(kThreads) tv_kernel(const __grid_constant__ TvArgs a, const float* __restrict__ P,
                                                      float* __restrict__ g, float* __restrict__ partial) {
  __shared__ float tmp[kThreads / 32];
  float acc = 0.f;
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < a.total;
       i += (long long)gridDim.x * kThreads) {
    int q = 0;
    long long rel = i;
    while (q + 1 < a.n_planes && rel >= a.p[q].cells) rel -= a.p[q++].cells;
    const TvPlane pl = a.p[q];
    const long long e = pl.off + rel;
    const long long cell = rel / a.h;
    const int ai = (int)(cell % pl.ra), bi = (int)(cell / pl.ra);
    const long long sa = a.h, sb = (long long)pl.ra * a.h;
    const float v = P[e];
    float gr = 0.f;
    if (ai + 1 < pl.ra) {
      const float d = P[e + sa] - v;
      acc += d * d * (0.5f * pl.wa);
      gr -= pl.wa * d;
    }
    if (ai > 0) gr += pl.wa * (v - P[e - sa]);
    if (bi + 1 < pl.rb) {
      const float d = P[e + sb] - v;
      acc += d * d * (0.5f * pl.wb);
      gr -= pl.wb * d;
    }
    if (bi > 0) gr += pl.wb * (v - P[e - sb]);
    g[e] += gr;
  }
  const float s = block_sum(acc, tmp);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Bias-corrected Adam over every segment; the gradient is cleared after use so the
// next step accumulates afresh.  Element i of a segment takes lr_head where
// (i mod period) < head (the degree-0 SH coefficients), else lr.
__global__ void __launch_bounds__(kThreads) adam_kernel(const __grid_constant__ AdamArgs a) {
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < a.total;
       i += (long long)gridDim.x * kThreads) {
    int q = 0;
    long long j = i;
    while (q + 1 < a.n_segs && j >= a.seg[q].n) j -= a.seg[q++].n;
    const AdamSeg& sgm = a.seg[q];
    const float lr = (sgm.period > 0 && (int)(j % sgm.period) < sgm.head) ? sgm.lr_head : sgm.lr;
    const float gv = sgm.g[j];
    const float m = a.beta1 * sgm.m[j] + (1.f - a.beta1) * gv;
    const float v = a.beta2 * sgm.v[j] + (1.f - a.beta2) * gv * gv;
    sgm.m[j] = m;
    sgm.v[j] = v;
    sgm.p[j] -= lr * (m / a.c1) / (sqrtf(v / a.c2) + a.eps);
    sgm.g[j] = 0.f;
  }
}

// Derived copies of the updated parameters: planes in BF16 (round to nearest
// even), and every MLP value into the transposed float32 layout and, where it has
// one, its place in the tensor-core operand image (BF16) or bias table.
__global__ void __launch_bounds__(kThreads) derive_kernel(const float* __restrict__ planes, long long n_planes,
                                                          __nv_bfloat16* __restrict__ planes_bf16,
                                                          const float* __restrict__ mlp, int n_mlp,
                                                          const int4* __restrict__ tab, float* __restrict__ mlp_t,
                                                          uint8_t* __restrict__ tc_ops, float* __restrict__ tc_bias) {
  const long long stride = (long long)gridDim.x * kThreads;
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n_planes; i += stride)
    planes_bf16[i] = __float2bfloat16_rn(planes[i]);
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n_mlp; i += stride) {
    const float v = mlp[i];
    const int4 d = tab[i];
    mlp_t[d.x] = v;
    if (tc_ops && d.y >= 0) *reinterpret_cast<__nv_bfloat16*>(tc_ops + d.y) = __float2bfloat16_rn(v);
    if (tc_bias && d.z >= 0) tc_bias[d.z] = v;
  }
}

int grid_for(long long n) {
  const long long want = (n + kThreads - 1) / kThreads;
  const long long cap = 4LL * device_sm_count();
  return (int)std::max(1LL, std::min(want, cap));
}

}  // namespace

int train_partials() { return 4 * device_sm_count(); }

cudaError_t launch_l1(const float* img, const float* tgt, long long count, float* dl, float* partial, float* out,
                      cudaStream_t s) {
  if (count <= 0) return cudaErrorInvalidValue;
  const int grid = grid_for((count + 3) / 4);
  const bool aligned = ((reinterpret_cast<uintptr_t>(img) | reinterpret_cast<uintptr_t>(tgt) |
                         reinterpret_cast<uintptr_t>(dl)) & 15u) == 0;
  l1_kernel<<<grid, kThreads, 0, s>>>(img, tgt, count, aligned ? count / 4 : 0, (float)(1.0 / (double)count), dl,
                                      partial);
  finish_sum_kernel<<<1, kThreads, 0, s>>>(partial, grid, 1.0 / (double)count, out);
  return cudaGetLastError();
}

cudaError_t launch_tv(const PlaneGeom& pg, const float* planes, float weight, float* g_planes, float* partial,
                      float* out, cudaStream_t s) {
  TvArgs a{};
  a.h = pg.feat_dim;
  const int axes[6][2] = {{0, 1}, {0, 2}, {1, 2}, {0, 3}, {1, 3}, {2, 3}};
  long long total = 0;
  for (int l = 0; l < pg.n_levels; ++l)
    for (int p = 0; p < 6; ++p) {
      TvPlane& q = a.p[a.n_planes++];
      q.ra = axes[p][0] == 3 ? pg.res_time : pg.res[l];
      q.rb = axes[p][1] == 3 ? pg.res_time : pg.res[l];
      q.off = pg.off[l][p];
      q.cells = (long long)q.ra * q.rb * pg.feat_dim;
      const double na = (double)q.rb * (q.ra - 1) * pg.feat_dim, nb = (double)(q.rb - 1) * q.ra * pg.feat_dim;
      q.wa = (float)(2.0 * weight / na);
      q.wb = (float)(2.0 * weight / nb);
      total += q.cells;
    }
  a.total = total;
  const int grid = grid_for(total);
  tv_kernel<<<grid, kThreads, 0, s>>>(a, planes, g_planes, partial);
  finish_sum_kernel<<<1, kThreads, 0, s>>>(partial, grid, 1.0, out);
  return cudaGetLastError();
}

cudaError_t launch_adam(const AdamArgs& a, cudaStream_t s) {
  if (a.total <= 0) return cudaSuccess;
  adam_kernel<<<grid_for(a.total), kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_derive(const float* planes, long long n_planes, __nv_bfloat16* planes_bf16, const float* mlp,
                          int n_mlp, const int4* tab, float* mlp_t, uint8_t* tc_ops, float* tc_bias,
                          cudaStream_t s) {
  derive_kernel<<<grid_for(std::max<long long>(n_planes, n_mlp)), kThreads, 0, s>>>(
      planes, n_planes, planes_bf16, mlp, n_mlp, tab, mlp_t, tc_ops, tc_bias);
  return cudaGetLastError();
}

}  // namespace fs4d
