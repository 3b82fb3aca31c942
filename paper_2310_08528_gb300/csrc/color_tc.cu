// Colour and opacity heads (App. B) on the tensor cores, for the BF16 path: the
// heads of color.cu (C' = C + phi_C(f_d), logit' = logit + phi_alpha(f_d), each
// Lin(64 -> 64), ReLU, Lin(64 -> out)) as two GEMMs per tile of 128 Gaussians:
//   D1 [128 x 128] = F . [W_C1; W_a1]^T               both hidden layers (K = 64)
//   D2 [128 x 64]  = H . blockdiag(W_C2, W_a2)^T      3K colour outputs, then the
//                                                     opacity output (K = 128)
// F is f_d, which the BF16 deformation kernel leaves as each tile's operand image
// (BF16, UMMA canonical no-swizzle K-major layout, 16 KB per tile), H the ReLU'd
// hidden layers in BF16 in the same layout.  The outputs are staged in shared
// memory and written row by row, so that a warp's stores cover whole rows of C'.  Each CTA converts the four layers from the scene's float32 weights into
// operand images in its own shared memory once, so a weight update needs no
// refresh.  Persistent CTAs (two per SM, 256 TMEM columns each); one thread issues
// each GEMM and commits it to an mbarrier; every wait is bounded (on a timeout the
// CTA records kStatusTimeout, stops, frees its TMEM and returns).
#include <type_traits>

#include "tc_util.cuh"

namespace fs4d {
namespace {
using namespace tcu;

constexpr int kThreads = 256;
constexpr int kRows = kTcRows;
constexpr int kW = 64;
constexpr uint32_t kTmemCols = 256;
// shared memory: B1 [128 x 64], B2 [64 x 128], F [128 x 64], H [128 x 128] (BF16
// operand images), the biases (hidden 128, outputs 64), the mbarrier, two words
constexpr int kB1 = 0;
constexpr int kB2 = kB1 + 128 * 64 * 2;
constexpr int kF = kB2 + 64 * 128 * 2;
constexpr int kH = kF + 128 * 64 * 2;
constexpr int kBias = kH + 128 * 128 * 2;
constexpr int kMbar = kBias + (128 + 64) * 4;
constexpr int kSmem = kMbar + 16;

// 8 consecutive floats -> one 16-byte row of a core matrix
__device__ __forceinline__ uint4 pack8(const float (&v)[8]) {
  uint4 q;
  q.x = pack_bf16(v[0], v[1]);
  q.y = pack_bf16(v[2], v[3]);
  q.z = pack_bf16(v[4], v[5]);
  q.w = pack_bf16(v[6], v[7]);
  return q;
}

template <int K3>
__global__ void __launch_bounds__(kThreads, 2) color_tc_kernel(const ColorArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  float* sBias = reinterpret_cast<float*>(smem + kBias);
  uint64_t* sMbar = reinterpret_cast<uint64_t*>(smem + kMbar);
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(sMbar + 1);
  uint32_t* sFail = sTmem + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the source layout: W_C1 [64][64], b_C1, W_C2 [K3][64], b_C2, W_a1, b_a1, W_a2 [64], b_a2
  const float* w = a.weights;
  constexpr int c1w = 0, c1b = c1w + kW * kW, c2w = c1b + kW, c2b = c2w + K3 * kW, a1w = c2b + K3,
                a1b = a1w + kW * kW, a2w = a1b + kW, a2b = a2w + kW;
  // operand images of the four layers: each thread loads all its values first (every
  // load in flight at once), then converts and stores them; B1 and B2 have 1024
  // chunks of 8 values each, 4 per thread
  {
    float v[4][8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {  // B1: rows 0..63 W_C1, 64..127 W_a1 (K = 64)
      const int c = tid + kThreads * j, r = c >> 3, k0 = (c & 7) * 8;
      const float* src = w + (r < kW ? c1w + r * kW : a1w + (r - kW) * kW) + k0;
#pragma unroll
      for (int k = 0; k < 8; ++k) v[j][k] = __ldg(src + k);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = tid + kThreads * j, r = c >> 3, k0 = (c & 7) * 8;
      *reinterpret_cast<uint4*>(smem + kB1 + a_off(r, k0, 64)) = pack8(v[j]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {  // B2: W_C2 on K 0..63, W_a2 in row K3 on K 64..127, else 0
      const int c = tid + kThreads * j, r = c >> 4, k0 = (c & 15) * 8;
      const bool col = r < K3 && k0 < kW, op = r == K3 && k0 >= kW;
      const float* src = w + (col ? c2w + r * kW + k0 : a2w + k0 - kW);
#pragma unroll
      for (int k = 0; k < 8; ++k) v[j][k] = (col || op) ? __ldg(src + k) : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = tid + kThreads * j, r = c >> 4, k0 = (c & 15) * 8;
      *reinterpret_cast<uint4*>(smem + kB2 + a_off(r, k0, 128)) = pack8(v[j]);
    }
  }
  if (tid < 128 + 64) {
    const int i = tid;
    float b = 0.f;
    if (i < kW) b = __ldg(w + c1b + i);
    else if (i < 2 * kW) b = __ldg(w + a1b + i - kW);
    else if (i - 2 * kW < K3) b = __ldg(w + c2b + i - 2 * kW);
    else if (i - 2 * kW == K3) b = __ldg(w + a2b);
    sBias[i] = b;
  }
  const uint32_t mbar = smem_u32(sMbar);
  if (tid == 0) {
    mbar_init(mbar);
    *sFail = 0;
  }
  if (warp == 0) tmem_alloc(smem_u32(sTmem), kTmemCols);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  pdl_wait();  // f_d comes from the deformation kernel before this one
  pdl_trigger();
  const uint32_t tmem = *sTmem;
  const uint32_t s_addr = smem_u32(smem);
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const int row = (warp & 3) * 32 + lane;  // accumulator row (TMEM lane) this thread reads back
  const int half = warp >> 2;              // which half of the columns
  uint32_t phase = 0;
  const long long tiles = ((long long)a.n + kRows - 1) / kRows;
  // C' rows of a tile, cooperatively: vector q (kVec floats) of row r is item r * kPerRow + q
  constexpr int kVec = (K3 % 4 == 0) ? 4 : 1;
  constexpr int kPerRow = K3 / kVec;
  constexpr int kItems = (kRows * kPerRow + kThreads - 1) / kThreads;
  constexpr int kStride = K3 + 1;  // staged row: K3 colour offsets, then the opacity offset
  float* sOut = reinterpret_cast<float*>(smem + kH);  // reuses H once D2 has read it
  static_assert(kRows * kStride * 4 <= 128 * 128 * 2, "staged outputs fit in H");
  // this tile's F image, and the next tile's while this one's GEMMs run (4 x 16 B per thread)
  uint4 fimg[4];
  auto load_f = [&](long long t) {
    const uint4* src = a.fd_tiles + (size_t)t * (kRows * 64 / 8);
#pragma unroll
    for (int j = 0; j < 4; ++j) fimg[j] = __ldg(src + tid + kThreads * j);
  };
  if (blockIdx.x < tiles) load_f(blockIdx.x);
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long long base = tile * kRows;
#pragma unroll
    for (int j = 0; j < 4; ++j) reinterpret_cast<uint4*>(smem + kF)[tid + kThreads * j] = fimg[j];
    fence_async_smem();
    __syncthreads();
    // ---- D1 (cols 0..127) = F . [W_C1; W_a1]^T -> H = relu(D1 + b) in BF16
    if (tid == 0) {
      tc_fence_after();
      issue_gemm(tmem, 0, s_addr + kF, s_addr + kB1, 64, 128, mbar);
    }
    if (tile + gridDim.x < tiles) load_f(tile + gridDim.x);
    // the canonical colours this thread will write, and its row's opacity logit, loaded
    // while the GEMMs run
    using V = typename std::conditional<kVec == 4, float4, float>::type;
    V cs[kItems];
    int gi[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
      const int it = tid + kThreads * j, r = it / kPerRow, q = it % kPerRow;
      const bool ok = it < kRows * kPerRow && base + r < a.n;
      gi[j] = ok ? (a.perm ? (int)__ldg(a.perm + base + r) : (int)(base + r)) : -1;
      if (ok) cs[j] = __ldg(reinterpret_cast<const V*>(a.sh + (size_t)gi[j] * K3) + q);
    }
    int g_row = -1;
    float logit = 0.f;
    if (tid < kRows && base + tid < a.n) {
      g_row = a.perm ? (int)__ldg(a.perm + base + tid) : (int)(base + tid);
      logit = __ldg(a.logits + g_row);
    }
    if (!mbar_wait(mbar, phase)) *sFail = 1;
    phase ^= 1;
    tc_fence_after();
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      float v[32];
      const int c0 = half * 64 + 32 * j;
      tmem_ld32(tmem + lane_base + (uint32_t)c0, v);
      store_relu32(smem + kH, row, c0, 128, v, sBias + c0);
    }
    tc_fence_before();
    fence_async_smem();
    __syncthreads();
    // ---- D2 (cols 128..191) = H . blockdiag(W_C2, W_a2)^T -> staged offsets
    if (tid == 0) {
      tc_fence_after();
      issue_gemm(tmem, 128, s_addr + kH, s_addr + kB2, 128, 64, mbar);
    }
    if (!mbar_wait(mbar, phase)) *sFail = 1;
    phase ^= 1;
    tc_fence_after();
    {
      float v[32];
      tmem_ld32(tmem + lane_base + 128u + (uint32_t)(half * 32), v);
      const float* b = sBias + 128 + half * 32;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (half * 32 + j <= K3) sOut[row * kStride + half * 32 + j] = v[j] + b[j];
    }
    __syncthreads();
    // ---- C' = C + offset, whole rows per warp; logit' = logit + offset
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
      if (gi[j] < 0) continue;
      const int it = tid + kThreads * j, r = it / kPerRow, q = it % kPerRow;
      const float* o = sOut + r * kStride + q * kVec;
      V out = cs[j];
      if constexpr (kVec == 4) {
        out.x += o[0];
        out.y += o[1];
        out.z += o[2];
        out.w += o[3];
      } else {
        out += o[0];
      }
      reinterpret_cast<V*>(a.sh_out + (size_t)gi[j] * K3)[q] = out;
    }
    if (g_row >= 0) a.logit_out[g_row] = logit + sOut[tid * kStride + K3];
    tc_fence_before();
    __syncthreads();
    if (*sFail) break;  // uniform: read after the barrier
  }
  tc_fence_after();
  if (*sFail && tid == 0 && a.status) atomicOr(a.status, kStatusTimeout);
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

template <int K3>
cudaError_t launch_k(const ColorArgs& a, cudaStream_t s) {
  static PerDeviceFlag attr;
  cudaError_t e = once_per_device(attr, [] {
    return cudaFuncSetAttribute(color_tc_kernel<K3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  });
  if (e != cudaSuccess) return e;
  const long long tiles = ((long long)a.n + kRows - 1) / kRows;
  const int sms = device_sm_count();
  const int grid = (int)(tiles < 2LL * sms ? tiles : 2LL * sms);
  return launch_pdl(color_tc_kernel<K3>, grid, kThreads, kSmem, s, a);
}

}  // namespace

cudaError_t launch_color_heads_bf16(const ColorArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (!a.fd_tiles || (reinterpret_cast<uintptr_t>(a.fd_tiles) & 15u) || (reinterpret_cast<uintptr_t>(a.sh) & 15u) ||
      (reinterpret_cast<uintptr_t>(a.sh_out) & 15u))
    return cudaErrorInvalidValue;
  switch (a.k3) {
    case 3: return launch_k<3>(a, s);
    case 12: return launch_k<12>(a, s);
    case 27: return launch_k<27>(a, s);
    case 48: return launch_k<48>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fs4d
