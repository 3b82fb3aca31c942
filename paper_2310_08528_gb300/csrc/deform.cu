// Gaussian deformation field, float32 SIMT path (Sec. 4.2, Eq. 5, Eq. 6).
//
// Persistent 256-thread CTAs (one per SM) walk tiles of 128 Gaussians.  Per tile:
//   1. Eq. 5: normalise (x, y, z) by the scene box and t to [-1, 1], bilinearly
//      interpolate the six planes xy xz yz xt yt zt of every level and multiply
//      them channel-wise.  h/4 consecutive lanes share one (Gaussian, level) item
//      and each owns one float4 of features, so a warp's loads cover whole grid
//      vertices (channels-last) with many requests in flight per thread;
//   2. phi_d (two ReLU layers) and the three heads as register-blocked SIMT
//      GEMMs: thread (warp w, lane l) computes outputs 8w..8w+7 of Gaussians
//      4l..4l+3, so one 128-bit activation load and two broadcast 128-bit weight
//      loads feed 32 FMAs.  Every output keeps the order b + sum_i w_i x_i of a
//      plain dot product;
//   3. Eq. 6: add the deltas to X, r, s.
// Activations live feature-major in shared memory ([feature][132]: 128 Gaussians
// plus 4 floats of padding, which keeps both access patterns conflict-free); the
// MLP is kept transposed (Wt[in][out]).
#include "fs4d_internal.cuh"

namespace fs4d {
namespace {


__device__ __forceinline__ void axis_setup(float u, int R, int& i0, float& f) {
  const float uc = fminf(1.f, fmaxf(-1.f, u));
  const float g = (uc + 1.f) * 0.5f * (float)(R - 1);
  int i = (int)floorf(g);
  i = max(0, min(i, R - 2));
  i0 = i;
  f = g - (float)i;
}

constexpr int kThreads = 256;
constexpr int kTileG = 128;          // Gaussians per tile
constexpr int kGS = kTileG + 4;      // row stride of the activation arrays (floats)

// acc[g][o] = b[o8 + o] + sum_i Wt[i][o8 + o] * src[i][g4 + g], in input order.
template <int IN>
__device__ __forceinline__ void layer64(const float* __restrict__ Wt, const float* __restrict__ b,
                                        const float* __restrict__ src, int g4, int o8, float (&acc)[4][8]) {
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    const float bo = b[o8 + o];
#pragma unroll
    for (int g = 0; g < 4; ++g) acc[g][o] = bo;
  }
  // outputs in pairs: one f32x2 FMA per two outputs (each element the same FP32 FMA)
  float2 a2[4][4];
#pragma unroll
  for (int g = 0; g < 4; ++g)
#pragma unroll
    for (int o = 0; o < 4; ++o) a2[g][o] = make_float2(acc[g][2 * o], acc[g][2 * o + 1]);
#pragma unroll 4
  for (int i = 0; i < IN; ++i) {
    const float4 x = *reinterpret_cast<const float4*>(src + i * kGS + g4);
    const float4 w0 = *reinterpret_cast<const float4*>(Wt + i * kWidth + o8);
    const float4 w1 = *reinterpret_cast<const float4*>(Wt + i * kWidth + o8 + 4);
    const float xs[4] = {x.x, x.y, x.z, x.w};
    const float2 ws[4] = {make_float2(w0.x, w0.y), make_float2(w0.z, w0.w), make_float2(w1.x, w1.y),
                          make_float2(w1.z, w1.w)};
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const float2 xg = make_float2(xs[g], xs[g]);
#pragma unroll
      for (int o = 0; o < 4; ++o) a2[g][o] = __ffma2_rn(ws[o], xg, a2[g][o]);
    }
  }
#pragma unroll
  for (int g = 0; g < 4; ++g)
#pragma unroll
    for (int o = 0; o < 4; ++o) {
      acc[g][2 * o] = a2[g][o].x;
      acc[g][2 * o + 1] = a2[g][o].y;
    }
}

__device__ __forceinline__ void store_relu(float* __restrict__ dst, int g4, int o8, const float (&acc)[4][8]) {
#pragma unroll
  for (int o = 0; o < 8; ++o)
    *reinterpret_cast<float4*>(dst + (o8 + o) * kGS + g4) =
        make_float4(fmaxf(acc[0][o], 0.f), fmaxf(acc[1][o], 0.f), fmaxf(acc[2][o], 0.f), fmaxf(acc[3][o], 0.f));
}

// Output layer of one head: D[off + j][g] = b2[j] + sum_o W2[o][j] * hid[o][g].
template <int OUT>
__device__ __forceinline__ void head_out(const float* __restrict__ W2, const float* __restrict__ b2,
                                         const float* __restrict__ hid, float* __restrict__ D, int off) {
  for (int j = threadIdx.x; j < OUT * kTileG; j += kThreads) {
    const int g = j % kTileG, oo = j / kTileG;
    float s = b2[oo];
#pragma unroll 8
    for (int o = 0; o < kWidth; ++o) s = fmaf(W2[o * OUT + oo], hid[o * kGS + g], s);
    D[(off + oo) * kGS + g] = s;
  }
}

template <int H, int L>
__global__ void __launch_bounds__(kThreads, 1) deform_fp32_kernel(DeformArgs a) {
  constexpr int HL = H * L;
  constexpr int XR = HL > kWidth ? HL : kWidth;
  constexpr int Q = H / 4;  // float4 groups per grid vertex
  extern __shared__ float4 smem4[];
  float* sw = reinterpret_cast<float*>(smem4);
  float* X = sw + a.mg.total;   // [XR][kGS]: f_h, then a1, then f_d (in place)
  float* Hd = X + XR * kGS;     // [64][kGS]: hidden layer of the current head
  float* D = Hd + kWidth * kGS; // [10][kGS]: deltas
  // the tile's rows: (X, t), quaternion, (log-scales, Gaussian index as bits)
  float4* sRowX = reinterpret_cast<float4*>(D + kDeltaDim * kGS);
  float4* sRowQ = sRowX + kTileG;
  float4* sRowS = sRowQ + kTileG;
  // the weights by cp.async (every 16-byte copy in flight at once), waited for
  // before the first tile's MLP below
  for (int i = threadIdx.x; i < a.mg.total / 4; i += kThreads) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem4 + i);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(reinterpret_cast<const float4*>(a.mlp_t) + i)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  // the weights above are the scene's; the rows below may come from earlier work
  pdl_wait();
  pdl_trigger();
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < a.zero_n16; i += (long long)gridDim.x * kThreads)
    a.zero[i] = make_uint4(0u, 0u, 0u, 0u);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g4 = lane * 4, o8 = warp * 8;
  const PlaneGeom& pg = a.pg;
  const MlpGeomT& mg = a.mg;
  const long long total = (long long)a.n * a.n_t;
  const long long tiles = (total + kTileG - 1) / kTileG;
  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long long base = tile * kTileG;
    __syncthreads();  // weights loaded / the previous tile fully written out
    // ---- 0. the tile's rows gathered once into shared memory (the work-order
    // index, then position, t, quaternion and log-scales in one round of loads)
    if (threadIdx.x < kTileG) {
      const long long gi = base + threadIdx.x;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f), q4 = x, sc = x;
      if (gi < total) {
        const int ti = (int)(gi / a.n);
        const int gw = (int)(gi - (long long)ti * a.n);
        const int g = a.perm ? (int)a.perm[gw] : gw;  // spatially coherent work order
        const float t = a.ts ? a.ts[ti] : a.t0;
        x = make_float4(a.means[3 * g], a.means[3 * g + 1], a.means[3 * g + 2], t);
        q4 = reinterpret_cast<const float4*>(a.quats)[g];
        sc = make_float4(a.log_scales[3 * g], a.log_scales[3 * g + 1], a.log_scales[3 * g + 2], __int_as_float(g));
      }
      sRowX[threadIdx.x] = x;
      sRowQ[threadIdx.x] = q4;
      sRowS[threadIdx.x] = sc;
    }
    __syncthreads();
    // ---- 1. Eq. 5 into X[0..HL)
    for (int item = threadIdx.x; item < kTileG * L * Q; item += kThreads) {
      const int q = item % Q, rl = item / Q;
      const int r = rl % kTileG, l = rl / kTileG;
      const long long gi = base + r;
      float f[4] = {0.f, 0.f, 0.f, 0.f};
      if (gi < total) {
        const float4 xr = sRowX[r];
        float c[4];
        c[0] = (xr.x - pg.aabb_min[0]) * pg.aabb_scale[0] - 1.f;
        c[1] = (xr.y - pg.aabb_min[1]) * pg.aabb_scale[1] - 1.f;
        c[2] = (xr.z - pg.aabb_min[2]) * pg.aabb_scale[2] - 1.f;
        c[3] = 2.f * xr.w - 1.f;
        f[0] = f[1] = f[2] = f[3] = 1.f;
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
          const float4* v00 =
              reinterpret_cast<const float4*>(a.planes + pg.off[l][p] + ((long long)j0 * Ra + i0) * H) + q;
          const float4 A = __ldg(v00), B = __ldg(v00 + Q), C = __ldg(v00 + (long long)Ra * Q),
                       E = __ldg(v00 + (long long)Ra * Q + Q);
          const float w00 = (1.f - fa) * (1.f - fb), w10 = fa * (1.f - fb), w01 = (1.f - fa) * fb, w11 = fa * fb;
          f[0] *= w00 * A.x + w10 * B.x + w01 * C.x + w11 * E.x;
          f[1] *= w00 * A.y + w10 * B.y + w01 * C.y + w11 * E.y;
          f[2] *= w00 * A.z + w10 * B.z + w01 * C.z + w11 * E.z;
          f[3] *= w00 * A.w + w10 * B.w + w01 * C.w + w11 * E.w;
        }
      }
      // rows 4q..4q+3 of column r; the store order is rotated by q/2 so that the
      // lanes of one store hit 32 distinct banks
      float* dst = X + (l * H + 4 * q) * kGS + r;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int e = (s + (q >> 1)) & 3;
        const float v = e == 0 ? f[0] : (e == 1 ? f[1] : (e == 2 ? f[2] : f[3]));
        dst[e * kGS] = v;
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");  // the weights (first tile; later a no-op)
    __syncthreads();

    // ---- 2. phi_d, in place in X
    float acc[4][8];
    layer64<HL>(sw + mg.w[0], sw + mg.b[0], X, g4, o8, acc);
    __syncthreads();
    store_relu(X, g4, o8, acc);
    __syncthreads();
    layer64<kWidth>(sw + mg.w[1], sw + mg.b[1], X, g4, o8, acc);
    __syncthreads();
    store_relu(X, g4, o8, acc);
    __syncthreads();
    if (a.fd_out) {  // f_d for the colour and opacity heads, rows in work order
      for (int e = threadIdx.x; e < kTileG * kWidth; e += kThreads) {
        const int r = e / kWidth, k = e - r * kWidth;
        if (base + r < total) a.fd_out[(size_t)(base + r) * kWidth + k] = X[k * kGS + r];
      }
    }
    // heads phi_x, phi_r, phi_s: hidden layer into Hd, output layer into D
    layer64<kWidth>(sw + mg.w[2], sw + mg.b[2], X, g4, o8, acc);
    store_relu(Hd, g4, o8, acc);
    __syncthreads();
    head_out<3>(sw + mg.w[3], sw + mg.b[3], Hd, D, 0);
    layer64<kWidth>(sw + mg.w[4], sw + mg.b[4], X, g4, o8, acc);
    __syncthreads();
    store_relu(Hd, g4, o8, acc);
    __syncthreads();
    head_out<4>(sw + mg.w[5], sw + mg.b[5], Hd, D, 3);
    layer64<kWidth>(sw + mg.w[6], sw + mg.b[6], X, g4, o8, acc);
    __syncthreads();
    store_relu(Hd, g4, o8, acc);
    __syncthreads();
    head_out<3>(sw + mg.w[7], sw + mg.b[7], Hd, D, 7);
    __syncthreads();

    // ---- 3. Eq. 6
    if (threadIdx.x < kTileG) {
      const int r = threadIdx.x;
      const long long gi = base + r;
      if (gi < total) {
        const int ti = (int)(gi / a.n);
        const float4 xr = sRowX[r], qv = sRowQ[r], sr = sRowS[r];
        const int g = __float_as_int(sr.w);
        float d[kDeltaDim];
#pragma unroll
        for (int k = 0; k < kDeltaDim; ++k) d[k] = D[k * kGS + r];
        const long long o = a.out_tab ? g : (long long)ti * a.n + g;
        float* om = a.out_tab ? a.out_tab[3 * ti] : a.out_means;
        float* oq = a.out_tab ? a.out_tab[3 * ti + 1] : a.out_quats;
        float* os = a.out_tab ? a.out_tab[3 * ti + 2] : a.out_log_scales;
        om[3 * o + 0] = xr.x + d[0];
        om[3 * o + 1] = xr.y + d[1];
        om[3 * o + 2] = xr.z + d[2];
        reinterpret_cast<float4*>(oq)[o] = make_float4(qv.x + d[3], qv.y + d[4], qv.z + d[5], qv.w + d[6]);
        os[3 * o + 0] = sr.x + d[7];
        os[3 * o + 1] = sr.y + d[8];
        os[3 * o + 2] = sr.z + d[9];
      }
    }
  }
}

template <int H, int L>
cudaError_t launch_t(const DeformArgs& a, cudaStream_t s) {
  constexpr int HL = H * L;
  constexpr int XR = HL > kWidth ? HL : kWidth;
  const size_t smem = sizeof(float) * ((size_t)a.mg.total + (size_t)(XR + kWidth + kDeltaDim) * kGS) +
                      3 * kTileG * sizeof(float4);
  static PerDeviceFlag attr;
  cudaError_t e = once_per_device(attr, [&] {
    return cudaFuncSetAttribute(deform_fp32_kernel<H, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
  const int sms = device_sm_count();
  const long long total = (long long)a.n * a.n_t;
  const long long need = (total + kTileG - 1) / kTileG;
  const int grid = (int)(need < sms ? need : sms);
  return launch_pdl(deform_fp32_kernel<H, L>, grid, kThreads, smem, s, a);
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
