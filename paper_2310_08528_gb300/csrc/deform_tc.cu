// Gaussian deformation field, BF16 tensor-core path (Sec. 4.2, Eq. 5, Eq. 6).
//
// One persistent CTA of 512 threads per SM, holding 256 TMEM columns, walks tiles of
// 128 (timestamp, Gaussian) rows with two warp groups:
//   1. samplers (warps 0-7): fetch each tile's rows one tile ahead (cp.async), then
//      take (row, level) items; each interpolates the six BF16 planes of its level
//      bilinearly in FP32, multiplies them (Eq. 5) and stores its h features as BF16
//      straight into the A operand tile -- one slot of a two-slot ring in shared
//      memory (UMMA canonical no-swizzle K-major layout) -- and marks the slot full
//      on its mbarrier;
//   2. consumers (warps 8-15) wait for the slot, then run four GEMMs on tcgen05
//      (kind::f16, BF16 x BF16 -> FP32 in TMEM, M = 128):
//        D1 = A1 . W_d1^T  (N 64)            f_h  -> hidden
//        D2 = A2 . W_d2^T  (N 64)            hidden -> f_d
//        D3 = A3 . [W_x1; W_r1; W_s1]^T (N 192)  three head hidden layers at once
//        D4 = A4 . blockdiag(W_x2, W_r2, W_s2)^T (N 16, 10 used; one GEMM per head over its
//             own 64 columns of A4)
//      one elected thread issues each GEMM and commits it to an mbarrier; between
//      GEMMs the consumers read the accumulator back with tcgen05.ld, add the bias,
//      apply ReLU, round to BF16 and write the next A tile; the last epilogue adds
//      dX, dr, ds to X, r, s (Eq. 6), and the slot is marked empty for the samplers.
// For scenes with colour and opacity heads (App. B) each tile's f_d operand image
// (A3) is also copied out, whole, as the input of the heads' tensor-core kernel.
// Every wait on an mbarrier is bounded; on a timeout the group records
// kStatusTimeout, both groups leave their loops on the same decision (a barrier
// reduction), the CTA frees its TMEM and returns.
#include "tc_util.cuh"

namespace fs4d {
namespace {
using namespace tcu;

constexpr int kSampWarps = 8;                      // warps 0..7 sample the planes
constexpr int kSampThreads = kSampWarps * 32;
constexpr int kConsWarps = 8;                      // warps 8..15 issue the GEMMs and run the epilogues
constexpr int kConsThreads = kConsWarps * 32;
constexpr int kColParts = kConsWarps / 4;          // consumer warps per TMEM lane quarter
constexpr int kThreads = kSampThreads + kConsThreads;
static_assert(kSampWarps % 4 == 0 && kConsWarps % 4 == 0, "consumer warp w reads TMEM lanes 32 (w % 4) ..");
constexpr int kRows = 128;
constexpr uint32_t kTmemCols = 256;
constexpr int kXBytes = 48 * 1024;  // activation tiles (A1+A2, then A3, then A4)
constexpr int kBiasFloats = 336;

__device__ __forceinline__ void axis_setup(float u, int R, int& i0, float& f) {
  const float uc = fminf(1.f, fmaxf(-1.f, u));
  const float g = (uc + 1.f) * 0.5f * (float)(R - 1);
  int i = (int)floorf(g);
  i = max(0, min(i, R - 2));
  i0 = i;
  f = g - (float)i;
}

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes_is16) {
  const uint32_t d = smem_u32(smem);
  if (bytes_is16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem) : "memory");
}

// Row r = tid of a tile into the row buffers (rx: X and t, rq: quaternion, rs:
// log-scales and the Gaussian index as bits): the work-order index is loaded, the
// rows are copied by cp.async (waited for at the start of the tile that uses them).
__device__ __forceinline__ void fetch_rows(const DeformArgs& a, long long base, long long total, int tid, float4* rx,
                                           float4* rq, float4* rs) {
  const long long gi = base + tid;
  if (gi < total) {
    const int ti = (int)(gi / a.n);
    const int gw = (int)(gi - (long long)ti * a.n);
    const int g = a.perm ? (int)a.perm[gw] : gw;
    float* x = reinterpret_cast<float*>(rx + tid);
    float* sc = reinterpret_cast<float*>(rs + tid);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cp_async(x + k, a.means + 3 * (size_t)g + k, 0);
      cp_async(sc + k, a.log_scales + 3 * (size_t)g + k, 0);
    }
    cp_async(rq + tid, reinterpret_cast<const float4*>(a.quats) + g, 1);
    x[3] = a.ts ? a.ts[ti] : a.t0;
    sc[3] = __int_as_float(g);
  } else {
    rx[tid] = rq[tid] = rs[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int H, int L>
__global__ void __launch_bounds__(kThreads, 1) deform_tc_kernel(DeformArgs a) {
  constexpr int HL = H * L;
  constexpr int kA1 = ((kRows * HL * 2) + 1023) / 1024 * 1024;  // one A1 buffer
  extern __shared__ __align__(1024) uint8_t smem[];
  const MlpGeomTC& tg = a.tg;
  const int b_bytes = (tg.bytes + 1023) / 1024 * 1024;
  uint8_t* sB = smem;
  uint8_t* sA1 = smem + b_bytes;          // [2][kA1]: the samplers' ring
  uint8_t* sX = sA1 + 2 * kA1;            // A2, then A3, then A4 (the consumers' activations)
  float* sBias = reinterpret_cast<float*>(sX + kXBytes);
  uint64_t* sBar = reinterpret_cast<uint64_t*>(sBias + kBiasFloats);  // mma, full[2], empty[2]
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(sBar + 5);
  uint32_t* sFail = sTmem + 1;
  // the rows of three tiles: (X, t), quaternion, (log-scales, Gaussian index as bits)
  float4* sRows = reinterpret_cast<float4*>(sBar + 6);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the weights by cp.async: every 16-byte copy in flight at once
  for (int i = tid; i < tg.bytes / 16; i += kThreads) cp_async(sB + 16 * i, a.tc_ops + 16 * i, 1);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int i = tid; i < kBiasFloats; i += kThreads) sBias[i] = a.tc_bias[i];
  const uint32_t mma_bar = smem_u32(sBar), full0 = smem_u32(sBar + 1), empty0 = smem_u32(sBar + 3);
  if (tid == 0) {
    for (int i = 0; i < 5; ++i) mbar_init(smem_u32(sBar + i));
    *sFail = 0;
  }
  if (warp == kSampWarps) tmem_alloc(smem_u32(sTmem), kTmemCols);
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  // the prologue above reads only the scene's weights; the rows below may come
  // from earlier work on the stream
  pdl_wait();
  pdl_trigger();
  for (long long i = (long long)blockIdx.x * kThreads + tid; i < a.zero_n16; i += (long long)gridDim.x * kThreads)
    a.zero[i] = make_uint4(0u, 0u, 0u, 0u);
  const uint32_t tmem = *sTmem;
  const PlaneGeom& pg = a.pg;
  const long long total = (long long)a.n * a.n_t;
  const long long tiles = (total + kRows - 1) / kRows;
  volatile uint32_t* fail = sFail;

  if (warp < kSampWarps) {
    // ================= samplers: rows and HexPlane features of each tile into the ring
    const int st = tid;  // 0 .. kSampThreads-1
    if (st < kRows) fetch_rows(a, (long long)blockIdx.x * kRows, total, st, sRows, sRows + kRows, sRows + 2 * kRows);
    int it = 0;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
      const int b = it & 1, rs = it % 3;
      const long long base = tile * kRows;
      // A1[b] and the row slot of tile it - 2 are free once the consumers finished that tile
      if (it >= 2 && !mbar_wait(empty0 + 8 * b, (uint32_t)((it >> 1) - 1) & 1u)) *fail = 1;
      asm volatile("cp.async.wait_all;\n" ::: "memory");  // this tile's rows (fetched one tile ahead)
      if (group_sync_or(1, kSampThreads, *fail != 0)) break;  // (the same decision in every sampler)
      if (st < kRows && tile + gridDim.x < tiles) {
        float4* nx = sRows + 3 * kRows * ((it + 1) % 3);
        fetch_rows(a, (tile + gridDim.x) * kRows, total, st, nx, nx + kRows, nx + 2 * kRows);
      }
      const float4* sRowX = sRows + 3 * kRows * rs;
      uint8_t* A1 = sA1 + b * kA1;
      // HexPlane features (Eq. 5) -> A1 [128 x HL] BF16.  Four (H = 32) or two
      // (H = 16) consecutive lanes share one (Gaussian, level) item and each owns 8
      // features, so a warp's 16-byte loads cover whole 64-byte grid vertices of 8
      // Gaussians and few registers per plane keep many loads in flight.
      constexpr int Q = H / 8;
      for (int item = st; item < kRows * L * Q; item += kSampThreads) {
        const int q = item % Q, rl = item / Q;
        const int r = rl % kRows, l = rl / kRows;
        const long long gi = base + r;
        float f[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) f[k] = 0.f;
        if (gi < total) {
          const float4 xr = sRowX[r];
          float c[4];
          c[0] = (xr.x - pg.aabb_min[0]) * pg.aabb_scale[0] - 1.f;
          c[1] = (xr.y - pg.aabb_min[1]) * pg.aabb_scale[1] - 1.f;
          c[2] = (xr.z - pg.aabb_min[2]) * pg.aabb_scale[2] - 1.f;
          c[3] = 2.f * xr.w - 1.f;
#pragma unroll
          for (int k = 0; k < 8; ++k) f[k] = 1.f;
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
            const uint4* v00 =
                reinterpret_cast<const uint4*>(a.planes_bf16 + pg.off[l][p] + ((long long)j0 * Ra + i0) * H) + q;
            const uint4 A = __ldg(v00), B = __ldg(v00 + Q), C = __ldg(v00 + (long long)Ra * Q),
                        D = __ldg(v00 + (long long)Ra * Q + Q);
            const float w00 = (1.f - fa) * (1.f - fb), w10 = fa * (1.f - fb), w01 = (1.f - fa) * fb, w11 = fa * fb;
            const uint32_t wa[4] = {A.x, A.y, A.z, A.w}, wb[4] = {B.x, B.y, B.z, B.w},
                           wc[4] = {C.x, C.y, C.z, C.w}, wd[4] = {D.x, D.y, D.z, D.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              f[2 * e] *= w00 * bf_lo(wa[e]) + w10 * bf_lo(wb[e]) + w01 * bf_lo(wc[e]) + w11 * bf_lo(wd[e]);
              f[2 * e + 1] *= w00 * bf_hi(wa[e]) + w10 * bf_hi(wb[e]) + w01 * bf_hi(wc[e]) + w11 * bf_hi(wd[e]);
            }
          }
        }
        uint4 v;
        v.x = pack_bf16(f[0], f[1]);
        v.y = pack_bf16(f[2], f[3]);
        v.z = pack_bf16(f[4], f[5]);
        v.w = pack_bf16(f[6], f[7]);
        *reinterpret_cast<uint4*>(A1 + a_off(r, l * H + 8 * q, HL)) = v;
      }
      fence_async_smem();
      group_sync(1, kSampThreads);
      if (st == 0) mbar_arrive(full0 + 8 * b);
    }
  } else {
    // ================= consumers: the four GEMMs of each tile and their epilogues
    const int ct = tid - kSampThreads, cw = warp - kSampWarps;
    const uint32_t b_addr = smem_u32(sB), x_addr = smem_u32(sX);
    const uint32_t lane_base = (uint32_t)((cw & 3) * 32) << 16;
    const int row = (cw & 3) * 32 + lane;  // accumulator row this thread reads back
    const int half = cw >> 2;              // which part of the columns it handles (of kColParts)
    uint32_t phase = 0;
    int it = 0;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
      const int b = it & 1, rs = it % 3;
      const long long base = tile * kRows;
      if (!mbar_wait(full0 + 8 * b, (uint32_t)(it >> 1) & 1u)) *fail = 1;
      if (group_sync_or(2, kConsThreads, *fail != 0)) break;  // (the same decision in every consumer)
      tc_fence_after();
      // ---- phi_d layer 1: D1 (cols 0..63) = A1 . W_d1^T
      if (ct == 0) issue_gemm(tmem, 0, smem_u32(sA1 + b * kA1), b_addr + tg.b1_off, HL, 64, mma_bar);
      if (!mbar_wait(mma_bar, phase)) *fail = 1;
      phase ^= 1;
      tc_fence_after();
#pragma unroll
      for (int j = 0; j < 2 / kColParts; ++j) {
        float v[32];
        const int c0 = half * (64 / kColParts) + 32 * j;
        tmem_ld32(tmem + lane_base + (uint32_t)c0, v);
        store_relu32(sX, row, c0, 64, v, sBias + 0 + c0);
      }
      tc_fence_before();
      fence_async_smem();
      group_sync(2, kConsThreads);

      // ---- phi_d layer 2: D2 (cols 64..127) = A2 . W_d2^T  -> f_d in A3 (X offset 0)
      if (ct == 0) {
        tc_fence_after();
        issue_gemm(tmem, 64, x_addr, b_addr + tg.b2_off, 64, 64, mma_bar);
      }
      if (!mbar_wait(mma_bar, phase)) *fail = 1;
      phase ^= 1;
      tc_fence_after();
#pragma unroll
      for (int j = 0; j < 2 / kColParts; ++j) {
        float v[32];
        const int c0 = half * (64 / kColParts) + 32 * j;
        tmem_ld32(tmem + lane_base + 64u + (uint32_t)c0, v);
        store_relu32(sX, row, c0, 64, v, sBias + 64 + c0);
      }
      tc_fence_before();
      fence_async_smem();
      group_sync(2, kConsThreads);

      // ---- heads, hidden layers: D3 (cols 0..191) = A3 . [W_x1; W_r1; W_s1]^T -> A4 [128 x 192]
      if (ct == 0) {
        tc_fence_after();
        issue_gemm(tmem, 0, x_addr, b_addr + tg.b3_off, 64, 192, mma_bar);
      }
      if (a.fd_tiles) {  // f_d as this tile's BF16 operand image (the colour heads' input), while D3 runs
        const uint4* src = reinterpret_cast<const uint4*>(sX);
        uint4* dst = a.fd_tiles + (size_t)tile * (kRows * 64 / 8);
        for (int i = ct; i < kRows * 64 / 8; i += kConsThreads) dst[i] = src[i];
        group_sync(2, kConsThreads);  // every consumer has read A3 before the epilogue below overwrites it
      }
      if (!mbar_wait(mma_bar, phase)) *fail = 1;
      phase ^= 1;
      tc_fence_after();
#pragma unroll
      for (int j = 0; j < 6 / kColParts; ++j) {
        float v[32];
        const int c0 = half * (192 / kColParts) + 32 * j;
        tmem_ld32(tmem + lane_base + (uint32_t)c0, v);
        store_relu32(sX, row, c0, 192, v, sBias + 128 + c0);
      }
      tc_fence_before();
      fence_async_smem();
      group_sync(2, kConsThreads);

      // ---- heads, output layers: A4 . blockdiag(W_x2, W_r2, W_s2)^T as three GEMMs over the
      // heads' own 64 columns of A4 (cols 192, 208, 224): three independent chains of 4 MMAs
      // instead of one of 12; the block-diagonal zeros made the other heads' terms exact zeros
      if (ct == 0) {
        tc_fence_after();
#pragma unroll
        for (int h = 0; h < 3; ++h) issue_mmas(tmem, 192 + 16 * h, x_addr, b_addr + tg.b4_off, 192, 64 * h, 64, 16);
        mma_commit(mma_bar);
      }
      if (!mbar_wait(mma_bar, phase)) *fail = 1;
      phase ^= 1;
      tc_fence_after();
      if (cw < 4) {
        float v[16], vr[16], vs[16];
        tmem_ld16(tmem + lane_base + 192u, v);
        tmem_ld16(tmem + lane_base + 208u, vr);
        tmem_ld16(tmem + lane_base + 224u, vs);
#pragma unroll
        for (int j = 3; j < 7; ++j) v[j] = vr[j];
#pragma unroll
        for (int j = 7; j < 10; ++j) v[j] = vs[j];
        const long long gi = base + row;
        if (gi < total) {
          const float4* sRowX = sRows + 3 * kRows * rs;
          const int ti = (int)(gi / a.n);
          const float4 xr = sRowX[row], q = sRowX[kRows + row], sr = sRowX[2 * kRows + row];
          const int g = __float_as_int(sr.w);
          const float* bo = sBias + 320;
          const long long o = a.out_tab ? (long long)g : (long long)ti * a.n + g;
          float* om = a.out_tab ? a.out_tab[3 * ti] : a.out_means;
          float* oq = a.out_tab ? a.out_tab[3 * ti + 1] : a.out_quats;
          float* os = a.out_tab ? a.out_tab[3 * ti + 2] : a.out_log_scales;
          om[3 * o + 0] = xr.x + (v[0] + bo[0]);
          om[3 * o + 1] = xr.y + (v[1] + bo[1]);
          om[3 * o + 2] = xr.z + (v[2] + bo[2]);
          reinterpret_cast<float4*>(oq)[o] =
              make_float4(q.x + (v[3] + bo[3]), q.y + (v[4] + bo[4]), q.z + (v[5] + bo[5]), q.w + (v[6] + bo[6]));
          os[3 * o + 0] = sr.x + (v[7] + bo[7]);
          os[3 * o + 1] = sr.y + (v[8] + bo[8]);
          os[3 * o + 2] = sr.z + (v[9] + bo[9]);
        }
      }
      tc_fence_before();
      group_sync(2, kConsThreads);
      if (ct == 0) mbar_arrive(empty0 + 8 * b);  // A1[b] and the row slot are free again
    }
  }
  __syncthreads();
  tc_fence_after();
  asm volatile("cp.async.wait_all;\n" ::: "memory");  // a row prefetch of a tile not run (timeout)
  if (*fail && tid == 0) atomicOr(a.status, kStatusTimeout);
  __syncthreads();
  if (warp == kSampWarps) tmem_dealloc(tmem, kTmemCols);
}

template <int H, int L>
cudaError_t launch_t(const DeformArgs& a, cudaStream_t s) {
  constexpr int kA1 = ((kRows * H * L * 2) + 1023) / 1024 * 1024;
  const size_t smem = (size_t)((a.tg.bytes + 1023) / 1024 * 1024) + 2 * kA1 + kXBytes + kBiasFloats * 4 + 48 +
                      9 * kRows * 16;
  static PerDeviceFlag attr;
  cudaError_t e = once_per_device(attr, [&] {
    return cudaFuncSetAttribute(deform_tc_kernel<H, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
  const int sms = device_sm_count();
  const long long tiles = ((long long)a.n * a.n_t + kRows - 1) / kRows;
  const int grid = (int)(tiles < sms ? tiles : sms);
  return launch_pdl(deform_tc_kernel<H, L>, grid, kThreads, smem, s, a);
}

}  // namespace

bool deform_bf16_supported(int feat_dim, int n_levels) {
  return (feat_dim == 16 || feat_dim == 32) && n_levels >= 1 && n_levels <= 3;
}

cudaError_t launch_deform_bf16(const DeformArgs& a, cudaStream_t s) {
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
