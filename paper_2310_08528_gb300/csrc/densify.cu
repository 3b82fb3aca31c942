// Densification and pruning of the canonical Gaussians (App. A keeps the
// adaptive density control of 3D Gaussian splatting).  Every Gaussian takes one
// of four decisions -- removed, kept, kept and copied, split into two children
// -- from its view-space gradient statistics, its largest log-scale and its
// opacity logit, all compared in float32.  The new set is laid out as the kept
// Gaussians, the copies, the first children and the second children, each in
// the old order, so an output's place is a sum of prefix counts:
//   count_kernel   per 256-Gaussian block: the number of kept, copied and split
//                  Gaussians (__syncthreads_count)
//   scan_kernel    one CTA: exclusive scans of the three block counts and totals
//   map_kernel     each Gaussian writes its outputs' source index and kind
//                  (block-local ranks from warp ballots)
//   gather_kernel  every per-Gaussian array (parameters, Adam moments) gathered
//                  by source index in output order; moments of new Gaussians 0
//   child_kernel   the children: mu + R S z with z ~ N(0, I) given by the
//                  caller (a draw from N(mu, R S S^T R^T), Eq. 2), log-scales
//                  minus ln 1.6
//   morton_kernel  30-bit Morton codes of the new means in the scene box: keys
//                  of the deformation work order (sorted by the library's radix
//                  sort)
// Each is one streaming pass (HBM-bound); none is on a frame's path.
#include "fs4d_internal.cuh"

namespace fs4d {
namespace {

constexpr int kThreads = 256;

// 0 removed, 1 kept, 2 kept and copied, 3 split.
__device__ __forceinline__ int decide(const DensifyArgs& a, int i) {
  if (a.opacity[i] < a.prune_logit) return 0;
  const float v = a.visible[i];
  const float avg = v > 0.f ? __fdiv_rn(a.grad_sum[i], v) : 0.f;
  if (!(avg >= a.grad_threshold)) return 1;
  const float* s = a.log_scales + 3 * (size_t)i;
  const float smax = fmaxf(fmaxf(s[0], s[1]), s[2]);
  return smax > a.split_log_scale ? 3 : 2;
}

__global__ void __launch_bounds__(kThreads) count_kernel(const DensifyArgs a) {
  const int i = blockIdx.x * kThreads + threadIdx.x;
  const int d = i < a.n ? decide(a, i) : 0;
  const int keep = __syncthreads_count(d == 1 || d == 2);
  const int copy = __syncthreads_count(d == 2);
  const int split = __syncthreads_count(d == 3);
  if (threadIdx.x == 0) {
    a.block_off[blockIdx.x] = (uint32_t)keep;
    a.block_off[gridDim.x + blockIdx.x] = (uint32_t)copy;
    a.block_off[2 * gridDim.x + blockIdx.x] = (uint32_t)split;
  }
}

// In place: block_off[c][b] becomes the exclusive prefix of category c; totals[c]
// the sum.  One CTA walks the blocks in chunks of kThreads.
__global__ void __launch_bounds__(kThreads) scan_kernel(uint32_t* block_off, int nb, uint32_t* totals) {
  __shared__ uint32_t s[kThreads];
  for (int c = 0; c < 3; ++c) {
    uint32_t* x = block_off + (size_t)c * nb;
    uint32_t carry = 0;
    for (int b0 = 0; b0 < nb; b0 += kThreads) {
      const int b = b0 + threadIdx.x;
      const uint32_t v = b < nb ? x[b] : 0u;
      s[threadIdx.x] = v;
      __syncthreads();
      for (int d = 1; d < kThreads; d <<= 1) {  // Hillis-Steele inclusive scan
        const uint32_t add = threadIdx.x >= (unsigned)d ? s[threadIdx.x - d] : 0u;
        __syncthreads();
        s[threadIdx.x] += add;
        __syncthreads();
      }
      if (b < nb) x[b] = carry + s[threadIdx.x] - v;
      carry += s[kThreads - 1];
      __syncthreads();
    }
    if (threadIdx.x == 0) totals[c] = carry;
  }
}

// Rank of the calling thread among the block's threads with `pred` (exclusive),
// given a [kThreads / 32] shared array.
__device__ __forceinline__ uint32_t block_rank(bool pred, uint32_t* warp_cnt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t bal = __ballot_sync(0xffffffffu, pred);
  if (lane == 0) warp_cnt[warp] = __popc(bal);
  __syncthreads();
  uint32_t before = 0;
  for (int w = 0; w < warp; ++w) before += warp_cnt[w];
  __syncthreads();
  return before + __popc(bal & ((1u << lane) - 1u));
}

__global__ void __launch_bounds__(kThreads) map_kernel(const DensifyArgs a) {
  __shared__ uint32_t cnt[kThreads / 32];
  const int i = blockIdx.x * kThreads + threadIdx.x;
  const int d = i < a.n ? decide(a, i) : 0;
  const uint32_t rk = block_rank(d == 1 || d == 2, cnt);
  const uint32_t rc = block_rank(d == 2, cnt);
  const uint32_t rs = block_rank(d == 3, cnt);
  const int nb = gridDim.x;
  const uint32_t tk = a.totals[0], tc = a.totals[1], ts = a.totals[2];
  if (d == 1 || d == 2) {
    const uint32_t o = a.block_off[blockIdx.x] + rk;
    a.src[o] = i;
    a.kind[o] = 0;
  }
  if (d == 2) {
    const uint32_t o = tk + a.block_off[nb + blockIdx.x] + rc;
    a.src[o] = i;
    a.kind[o] = 1;
  }
  if (d == 3) {
    const uint32_t o = tk + tc + a.block_off[2 * nb + blockIdx.x] + rs;
    a.src[o] = i;
    a.kind[o] = 2;
    a.src[o + ts] = i;
    a.kind[o + ts] = 3;
  }
}

// out[o][k] = in[src[o]][k]; with zero_new, 0 where kind[o] != 0.
__global__ void __launch_bounds__(kThreads) gather_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                          const int32_t* __restrict__ src,
                                                          const int32_t* __restrict__ kind, long long total,
                                                          int width, bool zero_new) {
  for (long long e = blockIdx.x * (long long)kThreads + threadIdx.x; e < total;
       e += (long long)gridDim.x * kThreads) {
    const long long o = e / width;
    const int k = (int)(e - o * width);
    out[e] = (zero_new && kind[o] != 0) ? 0.f : in[(size_t)src[o] * width + k];
  }
}

__global__ void __launch_bounds__(kThreads) child_kernel(const ChildArgs a) {
  const long long o = a.first + blockIdx.x * (long long)kThreads + threadIdx.x;
  if (o >= a.end) return;
  const int i = a.src[o], c = a.kind[o] - 2;
  const float4 q4 = reinterpret_cast<const float4*>(a.quats)[i];
  const float qn = sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w), qi = 1.f / qn;
  const float w = q4.x * qi, x = q4.y * qi, y = q4.z * qi, z = q4.w * qi;
  const float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                         {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                         {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
  const float* nz = a.normals + 6 * (size_t)i + 3 * c;
  float sz[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) sz[k] = expf(a.log_scales[3 * (size_t)i + k]) * nz[k];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    a.out_means[3 * o + r] = a.means[3 * (size_t)i + r] + (R[r][0] * sz[0] + R[r][1] * sz[1] + R[r][2] * sz[2]);
    a.out_log_scales[3 * o + r] = a.log_scales[3 * (size_t)i + r] - 0.47000362924573558f;  // ln 1.6
  }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 1023u;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__global__ void __launch_bounds__(kThreads) morton_kernel(const float* __restrict__ means, int n, float3 lo,
                                                          float3 hi, unsigned long long* __restrict__ keys,
                                                          uint32_t* __restrict__ values) {
  const int g = blockIdx.x * kThreads + threadIdx.x;
  if (g >= n) return;
  const float l[3] = {lo.x, lo.y, lo.z}, h[3] = {hi.x, hi.y, hi.z};
  uint32_t q[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float u = __fdiv_rn(means[3 * (size_t)g + k] - l[k], h[k] - l[k]);
    q[k] = (uint32_t)fminf(1023.f, fmaxf(0.f, __fmul_rn(u, 1023.f)));
  }
  keys[g] = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
  values[g] = (uint32_t)g;
}

int blocks_for(long long n) { return (int)((n + kThreads - 1) / kThreads); }

}  // namespace

int densify_blocks(int n) { return blocks_for(n); }

cudaError_t launch_densify_plan(const DensifyArgs& a, cudaStream_t s) {
  const int nb = blocks_for(a.n);
  count_kernel<<<nb, kThreads, 0, s>>>(a);
  scan_kernel<<<1, kThreads, 0, s>>>(a.block_off, nb, a.totals);
  return cudaGetLastError();
}

cudaError_t launch_densify_map(const DensifyArgs& a, cudaStream_t s) {
  map_kernel<<<blocks_for(a.n), kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gather(const float* in, float* out, const int32_t* src, const int32_t* kind, long long n_out,
                          int width, bool zero_new, cudaStream_t s) {
  const long long total = n_out * width;
  if (total <= 0) return cudaSuccess;
  const long long cap = 8LL * device_sm_count();
  gather_kernel<<<(int)std::min<long long>(cap, blocks_for(total)), kThreads, 0, s>>>(in, out, src, kind, total,
                                                                                     width, zero_new);
  return cudaGetLastError();
}

cudaError_t launch_children(const ChildArgs& a, cudaStream_t s) {
  if (a.end <= a.first) return cudaSuccess;
  child_kernel<<<blocks_for(a.end - a.first), kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_morton(const float* means, int n, const float lo[3], const float hi[3], unsigned long long* keys,
                          uint32_t* values, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  morton_kernel<<<blocks_for(n), kThreads, 0, s>>>(means, n, make_float3(lo[0], lo[1], lo[2]),
                                                    make_float3(hi[0], hi[1], hi[2]), keys, values);
  return cudaGetLastError();
}

}  // namespace fs4d
