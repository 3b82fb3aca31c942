// EWA projection of the deformed Gaussians (Eq. 2, Eq. 3) with view-dependent
// SH colour.  One thread per Gaussian; the structure-of-arrays inputs are read
// with coalesced loads (quaternions as one 128-bit load) and every output is a
// coalesced store.  Every input load is issued at the start: the SH rows (the
// bulk of the bytes) go to shared memory by cp.async and are waited for only
// when the colour is evaluated, so their latency overlaps the geometry.  Float32
// throughout.
#include "fs4d_internal.cuh"

namespace fs4d {
namespace {

// Real SH normalisation constants (textbook real basis without the
// Condon-Shortley phase), degree-major, m = -l..l.
constexpr float kY00 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kY1 = 0.48860251190291992f;    // sqrt(3/(4 pi))
constexpr float kY2a = 1.0925484305920792f;    // sqrt(15/pi)/2
constexpr float kY20 = 0.31539156525252005f;   // sqrt(5/pi)/4
constexpr float kY22 = 0.54627421529603959f;   // sqrt(15/pi)/4
constexpr float kY33 = 0.59004358992664352f;   // sqrt(35/(2 pi))/4
constexpr float kY32 = 2.8906114426405538f;    // sqrt(105/pi)/2
constexpr float kY31 = 0.45704579946446572f;   // sqrt(21/(2 pi))/4
constexpr float kY30 = 0.37317633259011540f;   // sqrt(7/pi)/4
constexpr float kY32b = 1.4453057213202769f;   // sqrt(105/pi)/4

constexpr float kDilation = 0.3f;   // low-pass dilation added to the 2-D covariance
constexpr float kGuard = 1.3f;      // guard band of the perspective Jacobian

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y) {
  Y[0] = kY00;
  if (deg < 1) return;
  Y[1] = kY1 * y; Y[2] = kY1 * z; Y[3] = kY1 * x;
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kY2a * x * y;
  Y[5] = kY2a * y * z;
  Y[6] = kY20 * (3.f * zz - 1.f);
  Y[7] = kY2a * x * z;
  Y[8] = kY22 * (xx - yy);
  if (deg < 3) return;
  Y[9] = kY33 * y * (3.f * xx - yy);
  Y[10] = kY32 * x * y * z;
  Y[11] = kY31 * y * (5.f * zz - 1.f);
  Y[12] = kY30 * z * (5.f * zz - 3.f);
  Y[13] = kY31 * x * (5.f * zz - 1.f);
  Y[14] = kY32b * z * (xx - yy);
  Y[15] = kY33 * x * (xx - 3.f * yy);
}

// Byte histograms of the depth keys for the depth sort that follows: shared-
// memory counts aggregated per warp (__match_any_sync), one global atomic per
// non-empty bin.
__device__ __forceinline__ void depth_histogram(const ProjectArgs& a, int g, float pz) {
  __shared__ uint32_t s_hist[4][256];
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  const bool valid = g < a.n;
  const uint32_t bits = valid ? __float_as_uint(pz) : 0u;
  uint32_t lt;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const uint32_t d = valid ? (bits >> (8 * p)) & 255u : 256u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    if (d < 256u && (peers & lt) == 0) atomicAdd(&s_hist[p][d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) {
    const uint32_t v = (&s_hist[0][0])[i];
    if (v) atomicAdd(&a.depth_hist[i], v);
  }
}

// float4 per Gaussian of SH coefficients when a row is 16-byte aligned (K*3 % 4 == 0),
// else 0 (read directly)
template <int DEG>
__host__ __device__ constexpr int sh_vec4() {
  return (3 * (DEG + 1) * (DEG + 1)) % 4 == 0 ? 3 * (DEG + 1) * (DEG + 1) / 4 : 0;
}

template <int DEG>
__global__ void __launch_bounds__(256) project_kernel(ProjectArgs a) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  constexpr int SHQ = sh_vec4<DEG>();
  extern __shared__ float4 s_sh[];  // [SHQ][256]: the CTA's SH rows, conflict-free per q
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = g < a.n;
  if (SHQ > 0 && valid) {
    const float4* src = reinterpret_cast<const float4*>(a.sh + (long long)g * K * 3);
#pragma unroll
    for (int q = 0; q < SHQ; ++q) {
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_sh[q * 256 + threadIdx.x]);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src + q) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  CamParams c = a.cam;
  if (a.cam_dev) {
    const fs4d_camera* d = a.cam_dev;
    c.fx = d->fx; c.fy = d->fy; c.cx = d->cx; c.cy = d->cy; c.znear = d->znear;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 4; ++k) c.m[4 * r + k] = d->world_to_cam[4 * r + k];
  }
  pdl_wait();  // (the SH rows and the camera are inputs of the frame; the Gaussians come from the deformation)
  pdl_trigger();
  float X0 = 0.f, X1 = 0.f, X2 = 0.f, logit = 0.f, ls0 = 0.f, ls1 = 0.f, ls2 = 0.f;
  float4 q4 = make_float4(1.f, 0.f, 0.f, 0.f);
  if (valid) {
    X0 = a.means[3 * g];
    X1 = a.means[3 * g + 1];
    X2 = a.means[3 * g + 2];
    logit = a.opacity_logits[g];
    q4 = reinterpret_cast<const float4*>(a.quats)[g];
    ls0 = a.log_scales[3 * g];
    ls1 = a.log_scales[3 * g + 1];
    ls2 = a.log_scales[3 * g + 2];
  }
  const float px = c.m[0] * X0 + c.m[1] * X1 + c.m[2] * X2 + c.m[3];
  const float py = c.m[4] * X0 + c.m[5] * X1 + c.m[6] * X2 + c.m[7];
  const float pz = c.m[8] * X0 + c.m[9] * X1 + c.m[10] * X2 + c.m[11];
  if (a.depth_hist) depth_histogram(a, g, pz);  // the whole CTA takes part
  if (!valid) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    return;
  }
  const float opacity = 1.f / (1.f + expf(-logit));
  a.depth[g] = pz;
  if (a.depth_keys) {
    a.depth_keys[g] = __float_as_uint(pz);
    a.depth_vals[g] = a.index_base + (uint32_t)g;
  }
  a.radius[g] = 0;
  a.rect[g] = make_int4(0, 0, 0, 0);
  a.xy[g] = make_float2(0.f, 0.f);
  a.conic_opacity[g] = make_float4(0.f, 0.f, 0.f, opacity);
  a.rgb[3 * g] = 0.f;
  a.rgb[3 * g + 1] = 0.f;
  a.rgb[3 * g + 2] = 0.f;
  // (every exit below first waits for this thread's SH copies)
  if (!(pz > c.znear)) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    return;
  }

  // Sigma = R S S^T R^T (Eq. 2), R from the normalised quaternion, S = diag(exp(s)).
  const float qinv = 1.f / sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
  const float w = q4.x * qinv, x = q4.y * qinv, y = q4.z * qinv, z = q4.w * qinv;
  const float R00 = 1.f - 2.f * (y * y + z * z), R01 = 2.f * (x * y - w * z), R02 = 2.f * (x * z + w * y);
  const float R10 = 2.f * (x * y + w * z), R11 = 1.f - 2.f * (x * x + z * z), R12 = 2.f * (y * z - w * x);
  const float R20 = 2.f * (x * z - w * y), R21 = 2.f * (y * z + w * x), R22 = 1.f - 2.f * (x * x + y * y);
  const float s0 = expf(ls0), s1 = expf(ls1), s2 = expf(ls2);

  // Sigma' = J W Sigma W^T J^T (Eq. 3) with the perspective Jacobian at the mean.
  // With Sigma = (R S)(R S)^T this is A A^T for the 2x3 matrix A = J W R S, which
  // is how it is evaluated: the determinant then comes from the squared 2x2
  // minors of A (Cauchy-Binet) plus the dilation terms, and the eigenvalue gap
  // from ((a - c)/2)^2 + b^2 -- sums of squares, so no float32 cancellation for
  // thin Gaussians (ac - b^2 would lose ~a*c/det ulps).
  const float limx = kGuard * (float)c.guard_w / (2.f * c.fx), limy = kGuard * (float)c.guard_h / (2.f * c.fy);
  const float iz = 1.f / pz;
  const float tx = fminf(limx, fmaxf(-limx, px * iz)) * pz;
  const float ty = fminf(limy, fmaxf(-limy, py * iz)) * pz;
  const float J00 = c.fx * iz, J02 = -c.fx * tx * iz * iz;
  const float J11 = c.fy * iz, J12 = -c.fy * ty * iz * iz;
  // T = J W (2x3)
  const float T00 = J00 * c.m[0] + J02 * c.m[8], T01 = J00 * c.m[1] + J02 * c.m[9], T02 = J00 * c.m[2] + J02 * c.m[10];
  const float T10 = J11 * c.m[4] + J12 * c.m[8], T11 = J11 * c.m[5] + J12 * c.m[9], T12 = J11 * c.m[6] + J12 * c.m[10];
  // A = T R S (2x3)
  const float A00 = (T00 * R00 + T01 * R10 + T02 * R20) * s0, A01 = (T00 * R01 + T01 * R11 + T02 * R21) * s1,
              A02 = (T00 * R02 + T01 * R12 + T02 * R22) * s2;
  const float A10 = (T10 * R00 + T11 * R10 + T12 * R20) * s0, A11 = (T10 * R01 + T11 * R11 + T12 * R21) * s1,
              A12 = (T10 * R02 + T11 * R12 + T12 * R22) * s2;
  const float aa = A00 * A00 + A01 * A01 + A02 * A02;
  const float bb = A00 * A10 + A01 * A11 + A02 * A12;
  const float dd = A10 * A10 + A11 * A11 + A12 * A12;
  const float m01 = A00 * A11 - A01 * A10, m02 = A00 * A12 - A02 * A10, m12 = A01 * A12 - A02 * A11;
  const float ca = aa + kDilation, cb = bb, cc = dd + kDilation;
  const float det = (m01 * m01 + m02 * m02 + m12 * m12) + kDilation * (aa + dd) + kDilation * kDilation;
  if (!(det > 0.f)) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    return;
  }
  const float idet = 1.f / det;
  const float hd = 0.5f * (aa - dd);
  const float lmax = 0.5f * (ca + cc) + sqrtf(hd * hd + bb * bb);
  const int radius = (int)ceilf(3.f * sqrtf(lmax));
  const float u = c.fx * px * iz + c.cx, v = c.fy * py * iz + c.cy;
  const float fr = (float)radius;
  int x0 = (int)floorf((u - fr) * (1.f / kTile)), x1 = (int)floorf((u + fr) * (1.f / kTile)) + 1;
  int y0 = (int)floorf((v - fr) * (1.f / kTile)), y1 = (int)floorf((v + fr) * (1.f / kTile)) + 1;
  x0 = min(a.tiles_x, max(0, x0)); x1 = min(a.tiles_x, max(0, x1));
  y0 = min(a.tiles_y, max(0, y0)); y1 = min(a.tiles_y, max(0, y1));
  if (x1 <= x0 || y1 <= y0) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    return;
  }

  // View-dependent colour: SH along the direction from the camera centre.
  const float cpx = -(c.m[0] * c.m[3] + c.m[4] * c.m[7] + c.m[8] * c.m[11]);
  const float cpy = -(c.m[1] * c.m[3] + c.m[5] * c.m[7] + c.m[9] * c.m[11]);
  const float cpz = -(c.m[2] * c.m[3] + c.m[6] * c.m[7] + c.m[10] * c.m[11]);
  float dx = X0 - cpx, dy = X1 - cpy, dz = X2 - cpz;
  const float dinv = 1.f / sqrtf(dx * dx + dy * dy + dz * dz);
  dx *= dinv; dy *= dinv; dz *= dinv;
  float Y[16];
  sh_basis(DEG, dx, dy, dz, Y);
  // K*3 coefficients per Gaussian: from the shared-memory copy (16-byte aligned
  // rows), else read directly
  float shc[3 * K];
  const float* sh = a.sh + (long long)g * K * 3;
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  if (SHQ > 0) {
#pragma unroll
    for (int q = 0; q < SHQ; ++q) {
      const float4 v = s_sh[q * 256 + threadIdx.x];
      shc[4 * q] = v.x; shc[4 * q + 1] = v.y; shc[4 * q + 2] = v.z; shc[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 3 * K; ++q) shc[q] = __ldg(sh + q);
  }
  float r = 0.5f, gg = 0.5f, b = 0.5f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    r += Y[k] * shc[3 * k];
    gg += Y[k] * shc[3 * k + 1];
    b += Y[k] * shc[3 * k + 2];
  }
  a.rgb[3 * g] = fmaxf(0.f, r);
  a.rgb[3 * g + 1] = fmaxf(0.f, gg);
  a.rgb[3 * g + 2] = fmaxf(0.f, b);
  a.xy[g] = make_float2(u, v);
  a.conic_opacity[g] = make_float4(cc * idet, -cb * idet, ca * idet, opacity);
  a.radius[g] = radius;
  a.rect[g] = make_int4(x0, y0, x1, y1);
}

}  // namespace

template <int DEG>
cudaError_t launch_project_deg(const ProjectArgs& a, unsigned grid, cudaStream_t s) {
  constexpr size_t smem = 16 * 256 * (size_t)sh_vec4<DEG>();
  if (smem > 0) {  // (with the 4 KB of static histogram the total can pass the 48 KB default)
    static PerDeviceFlag attr;
    cudaError_t e = once_per_device(attr, [] {
      return cudaFuncSetAttribute(project_kernel<DEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (e != cudaSuccess) return e;
  }
  return launch_pdl(project_kernel<DEG>, grid, 256, smem, s, a);
}

cudaError_t launch_project(const ProjectArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((a.n + 255) / 256);
  switch (a.sh_degree) {
    case 0: return launch_project_deg<0>(a, grid, s);
    case 1: return launch_project_deg<1>(a, grid, s);
    case 2: return launch_project_deg<2>(a, grid, s);
    case 3: return launch_project_deg<3>(a, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fs4d
