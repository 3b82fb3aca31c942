// Internal declarations shared by the kernel translation units of libfs4d.so.
// Kernels are written for sm_103a (GB300); nothing here is part of the C ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "fs4d.h"

namespace fs4d {

constexpr int kTile = 16;          // screen tile edge (pixels); one CTA composites one tile
constexpr int kMaxLevels = 4;      // HexPlane resolution levels supported
constexpr int kWidth = 64;         // MLP hidden width supported by the kernels
constexpr int kDeltaDim = 10;      // dX (3) + dr (4) + ds (3)

// Device status word bits (sticky until fs4d_check_device_status).
constexpr uint32_t kStatusTimeout = 1u;   // a bounded spin gave up
constexpr uint32_t kStatusCapacity = 2u;  // more tile pairs than buffer capacity

// Programmatic dependent launch.  The kernels of a frame are launched with
// launch_pdl, so a kernel's CTAs may start while the previous kernel on the stream
// finishes.  Each such kernel calls pdl_wait() before it touches memory written by
// earlier work on the stream -- griddepcontrol.wait returns when the previous grid
// has completed and its writes are visible, and since that grid itself waited for
// its own predecessor, everything before it has completed too -- and then
// pdl_trigger(): its dependent may launch once every CTA of this grid has triggered
// or exited (triggering only after the wait keeps the look-ahead to one kernel).
// Without the launch attribute both are no-ops.  The attribute is set only for
// launches outside stream capture: it shortens the gaps between eagerly launched
// kernels, but CUDA graphs captured with it replayed slower on GB300 than plain
// graphs (measured: 195 vs 175 us per 800x800 frame).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Kernel launches issued through launch_pdl by the calling thread (the frame
// kernels all are): the render entry points report a frame's count from it.
extern thread_local unsigned long long g_kernel_launches;

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                              Args... args) {
  ++g_kernel_launches;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return cudaGetLastError();
  cfg.attrs = attr;
  cfg.numAttrs = cs == cudaStreamCaptureStatusNone ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Bounded spin limit for decoupled look-back waits (iterations of ~100 ns).  The
// limit a launch uses is an argument (SortWork::spin_limit, EmitArgs::spin_limit)
// so that a context can lower it to exercise the timeout path (fs4d_set_wait_limit).
constexpr uint32_t kSpinLimit = 1u << 22;

// Per-device launcher state: whether a kernel's dynamic shared-memory attribute
// has been set on a device (cudaFuncSetAttribute applies to the current device
// only), and the SM count of the current device.
constexpr int kMaxDevices = 64;
struct PerDeviceFlag {
  std::atomic<bool> done[kMaxDevices] = {};
};
// Runs set() once per device for the flag; returns its error, or success.
template <typename F>
inline cudaError_t once_per_device(PerDeviceFlag& f, F set) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (f.done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = set();  // two threads may both set it: the attribute is the same
  if (e == cudaSuccess) f.done[dev].store(true, std::memory_order_release);
  return e;
}
int device_sm_count();  // SMs of the current device (cached per device; >= 1)

// ---------------------------------------------------------------- HexPlane geometry
struct PlaneGeom {
  int n_levels;
  int feat_dim;            // h
  int res_time;
  int res[kMaxLevels];     // spatial resolution per level
  long long off[kMaxLevels][6];  // element offset of each plane (xy xz yz xt yt zt)
  float aabb_min[3];
  float aabb_scale[3];     // 2 / (max - min): u = (x - min) * scale - 1
};

// ---------------------------------------------------------------- FP32 MLP layout
// The FP32 kernel keeps every layer transposed, Wt[in][out] followed by b[out],
// in the order d1 d2 x1 x2 r1 r2 s1 s2, so one 128-bit shared-memory load feeds
// four output accumulators.
struct MlpGeomT {
  int hin;                 // h * L
  int w[8], b[8];          // float offsets of Wt and b of each layer
  int total;               // floats (padded to a multiple of 4)
};

// ---------------------------------------------------------------- BF16 tcgen05 MLP layout
// Operand images of the four GEMMs (bf16, UMMA canonical no-swizzle K-major
// layout: 8x8 core matrices of 128 contiguous bytes; see deform_tc.cu):
//   B1 = d1 [64 x hin], B2 = d2 [64 x 64], B3 = x1|r1|s1 stacked [192 x 64],
//   B4 = block-diagonal x2/r2/s2 padded to [16 x 192].
struct MlpGeomTC {
  int hin;
  int b1_off, b2_off, b3_off, b4_off;   // byte offsets inside the operand image
  int bytes;                            // total operand image bytes
  int bias_off[4];                      // float offsets of the biases (64, 64, 192, 16)
  int bias_total;
};

struct DeformArgs {
  int n;                        // Gaussians
  const uint32_t* perm;         // optional [n] work order (spatially coherent); outputs keep Gaussian order
  int n_t;                      // timestamps
  const float* ts;              // device [n_t], or NULL to use t0 (n_t must be 1)
  float t0;
  const float* means;           // [n][3]
  const float* quats;           // [n][4]
  const float* log_scales;      // [n][3]
  float* out_means;             // [n_t][n][3]
  float* out_quats;             // [n_t][n][4]
  float* out_log_scales;        // [n_t][n][3]
  float* const* out_tab;        // optional [n_t][3] device table: per-timestamp output bases
                                // (means [n][3], quats [n][4], log-scales [n][3]); overrides out_*
  const float* planes;          // float32 planes
  const __nv_bfloat16* planes_bf16;
  const float* mlp_t;           // FP32 transposed layout (MlpGeomT)
  MlpGeomT mg;
  const uint8_t* tc_ops;        // BF16 operand image (MlpGeomTC)
  const float* tc_bias;
  MlpGeomTC tg;
  PlaneGeom pg;
  uint32_t* status;
  float* fd_out;                // FP32 kernel, optional [n][64]: f_d (after phi_d) in work order (n_t must be 1)
  uint4* zero;                  // optional: zero_n16 16-byte words the kernel sets to 0 (a frame's counters
  long long zero_n16;           // and look-back tables, cleared here instead of by a separate memset)
  uint4* fd_tiles;              // BF16 kernel, optional: f_d of each tile of 128 work-order rows as its BF16
                                // operand image (UMMA no-swizzle K-major, 16 KB per tile; n_t must be 1)
};

// Colour and opacity heads (App. B, color.cu): per Gaussian from f_d in work order.
struct ColorArgs {
  int n;
  const uint32_t* perm;         // work order (NULL: index order)
  const float* fd;              // SIMT form: [n][64] work order, 16-byte aligned
  const uint4* fd_tiles;        // tensor-core form: BF16 operand images, 16 KB per tile of 128 rows
  const float* weights;         // the four layers c1 c2 a1 a2 in the source layout (W[out][in] then b)
  int k3;                       // 3 x SH coefficients per channel
  const float* sh;              // [n][K][3] canonical
  const float* logits;          // [n] canonical
  float* sh_out;                // [n][K][3] deformed
  float* logit_out;             // [n] deformed
  uint32_t* status;             // optional: kStatusTimeout if a bounded wait gave up (tensor-core form)
};
int color_layer_floats(int k3);
// float32 SIMT form (the FP32 path)
cudaError_t launch_color_heads(const ColorArgs& a, cudaStream_t s);
// BF16 tcgen05 form (the BF16 path): k3 in {3, 12, 27, 48}; fd_tiles, sh, sh_out 16-byte aligned
cudaError_t launch_color_heads_bf16(const ColorArgs& a, cudaStream_t s);

struct CamParams {
  int width, height;
  float fx, fy, cx, cy, znear;
  float m[12];                  // rows 0..2 of world_to_cam
  int guard_w, guard_h;         // image extent the Jacobian's guard band refers to (the whole
                                // frame's, also when this call renders one band of it)
};

struct ProjectArgs {
  int n;
  const float* means;           // [n][3]
  const float* quats;           // [n][4]
  const float* log_scales;      // [n][3]
  const float* opacity_logits;  // [n]
  const float* sh;              // [n][K][3]
  int sh_degree;
  CamParams cam;
  const fs4d_camera* cam_dev;   // if non-NULL, read the camera from device memory
  int tiles_x, tiles_y;
  float2* xy;
  float4* conic_opacity;
  float* rgb;
  float* depth;
  int* radius;
  int4* rect;
  unsigned long long* depth_keys;  // optional [n]: float bits of depth, for the depth sort
  uint32_t* depth_vals;            // optional [n]: Gaussian index (index_base + g)
  uint32_t index_base;             // index of this call's first Gaussian in the frame's set
  uint32_t* depth_hist;            // optional [4][256] (zeroed): byte histograms of the depth keys
};

// Tile-pair emission fused with the exclusive scan of per-Gaussian tile counts
// (decoupled look-back) and with the digit histograms of every radix pass.
struct EmitArgs {
  int n;
  const uint32_t* order;        // [n] Gaussian indices in emission order (NULL: index order)
  const uint32_t* order_alt;    // with order_sel: the order is here when *order_sel != 0
  const uint32_t* order_sel;
  const float* depth;
  const int4* rect;
  int tiles_x;
  long long capacity;           // pairs the key/value buffers hold
  unsigned long long* keys;     // [capacity]
  uint32_t* values;             // [capacity]
  uint32_t* offsets;            // [n] exclusive prefix of tile counts (kept for the backward)
  unsigned long long* lookback; // [parts] scan look-back words (zeroed)
  uint32_t* part_counter;       // zeroed
  uint32_t* num_pairs;          // out: K (clamped to 2^32-1)
  uint32_t* num_pairs_sort;     // out: K if K <= capacity, else 0 (what the sort may read)
  int report_overflow;          // set kStatusCapacity in *status when K > capacity
  uint32_t* tile_count;         // [n_tiles] (zeroed): pairs per tile
  int n_tiles;
  uint32_t* status;
  uint32_t spin_limit;          // polls of the look-back wait before it gives up
  int packed;                   // 1: keys = (tile << 32) | Gaussian index, no values (the pairs
                                // are sorted on the tile bits only and the index travels along)
  // tile bitmap binning (launch_mark_tiles / launch_extract_tiles)
  uint32_t* bitmap;             // [n_tiles][words], bit (i & 31) of word i >> 5 of row t: the
                                // Gaussian of depth rank i touches tile t (all zero between frames)
  int words;                    // words per row: bitmap_words(n)
  const uint2* ranges;          // [n_tiles] tile [start, end) from the tile scan
  const uint32_t* tile_order;   // NULL or a permutation of the tiles: extraction order
  // with sorted_xy non-NULL, mark also copies the projected Gaussians into depth-rank order
  const float2* xy;
  const float4* conic_opacity;
  const float* rgb;
  float2* sorted_xy;            // [n]
  float4* sorted_co;            // [n]
  float* sorted_rgb;            // [n][3]
  int cull;                     // 1 (mark): set a bit only for the tiles whose pixel centres the
                                // Gaussian's ellipse {alpha >= 1/255} can reach.  The lists lose
                                // Gaussians no pixel of the tile blends: the image is unchanged,
                                // list positions are not the full rectangles'.
};

struct SortWork {
  uint32_t* hist;               // [8][256]
  uint32_t* lookback;           // [passes][max_parts][256]
  uint32_t* part_counters;      // [2 * 8 + 1]: pass tickets, then selection words
  long long max_parts;          // >= sort_parts(n_bound) lets every partition size be chosen
  bool prezeroed = false;       // tickets, selection words and look-back already zero
  uint32_t spin_limit = kSpinLimit;  // polls of a look-back wait before it gives up
  uint32_t* grid_counter = nullptr;  // optional, zero (with prezeroed): lets a small sort with result_sel
                                     // run every pass in one launch, its CTAs meeting at a grid barrier
};

// ---------------------------------------------------------------- launchers
cudaError_t launch_deform_fp32(const DeformArgs& a, cudaStream_t s);
cudaError_t launch_deform_bf16(const DeformArgs& a, cudaStream_t s);
bool deform_fp32_supported(int feat_dim, int n_levels);
bool deform_bf16_supported(int feat_dim, int n_levels);

cudaError_t launch_project(const ProjectArgs& a, cudaStream_t s);

int emit_parts(int n);          // scan partitions of the emit kernel
// keys[i] = float bits of depth[i] (upper word 0), vals[i] = i: input of the depth sort
cudaError_t launch_depth_keys(const float* depth, int n, unsigned long long* keys, uint32_t* vals, cudaStream_t s);
cudaError_t launch_scan_emit(const EmitArgs& a, cudaStream_t s);
// tile ranges (from the per-tile counts; all (0, 0) when num_pairs[1] == 0 < num_pairs[0]),
// if hist != NULL the [passes][256] digit histograms of the pair sort on the tile bits, and
// if order != NULL a permutation of the tiles, longest lists first (compositing launch order)
// capacity >= 0: the overflow test is the tiles' total > capacity instead (num_pairs[1] is then
// written as the total, or 0 on overflow, and status, if non-NULL, gets kStatusCapacity)
cudaError_t launch_tile_scan(const uint32_t* tile_count, int n_tiles, uint32_t* num_pairs, uint2* ranges,
                             uint32_t* hist, int passes, uint32_t* order, cudaStream_t s, long long capacity = -1,
                             uint32_t* status = nullptr);
// Tile bitmap binning (the alternative to emission + pair sort when the bitmap is small):
// mark sets the bit of every (tile, depth rank) pair and counts the pairs per tile
// (tile_count, num_pairs[0]); after the tile scan, extract walks each tile's row in rank
// order, writes the depth ranks at the tile's range -- or with ids the Gaussians (and
// keys if non-NULL) -- and clears the row.
int bitmap_words(int n);        // words per tile row (a multiple of 4)
cudaError_t launch_mark_tiles(const EmitArgs& a, cudaStream_t s);
cudaError_t launch_extract_tiles(const EmitArgs& a, bool ids, cudaStream_t s);

int sort_passes(int key_bits);
long long sort_parts(long long n);
// Stable LSD sort of (keys, values) on bits [first_bit, first_bit + key_bits).  n_dev (if non-NULL)
// holds the live count on the device; n_bound is an upper bound used to size the
// grids.  hist_ready = the per-pass histograms are already in work.hist.  Returns
// in *result_in_alt whether the sorted pairs ended in the alternate buffers.  With
// result_sel non-NULL, a pass whose digit is the same for every key copies nothing
// and the side that holds the result is known only on the device: *result_sel then
// points to a word that is 1 when it is the alternate buffers (*result_in_alt = false).
// work.part_counters must have 2 * 8 + 1 words.
cudaError_t launch_sort(unsigned long long* keys, uint32_t* values, unsigned long long* keys_alt,
                        uint32_t* values_alt, const uint32_t* n_dev, long long n_bound, int first_bit,
                        int key_bits, bool hist_ready, const SortWork& work, uint32_t* status, cudaStream_t s,
                        bool* result_in_alt, const uint32_t** result_sel = nullptr);
// order (optional): CTA i composites tile order[i]; values_stride: 1 for a list of
// uint32 indices, 2 for the low words of packed (tile | index) 64-bit keys
cudaError_t launch_composite(int width, int height, const uint2* ranges, const uint32_t* values,
                             const float2* xy, const float4* conic_opacity, const float* rgb, float* image,
                             float* t_final, int* n_contrib, cudaStream_t s, const uint32_t* order = nullptr,
                             int values_stride = 1);
}  // namespace fs4d

// ================================================================ training step
namespace fs4d {
// One Adam parameter segment: p -= lr m^ / (sqrt(v^) + eps), element i with
// (i mod period) < head takes lr_head (period 0: every element takes lr).
struct AdamSeg {
  float* p;
  float* g;
  float* m;
  float* v;
  long long n;
  float lr, lr_head;
  int period, head;
};
struct AdamArgs {
  AdamSeg seg[8];
  int n_segs;
  long long total;
  float beta1, beta2, eps;
  float c1, c2;   // bias corrections 1 - beta^step
};
int train_partials();  // size of the loss-partial buffers the launchers below need
// L1 loss: dl = sign(img - tgt) / count, *out = mean |img - tgt| (device float)
cudaError_t launch_l1(const float* img, const float* tgt, long long count, float* dl, float* partial, float* out,
                      cudaStream_t s);
// grid TV loss of the planes: g_planes += gradient, *out = loss
cudaError_t launch_tv(const PlaneGeom& pg, const float* planes, float weight, float* g_planes, float* partial,
                      float* out, cudaStream_t s);
cudaError_t launch_adam(const AdamArgs& a, cudaStream_t s);
// derived copies from planes and the source-layout MLP; tab[i] = (mlp_t index,
// tc_ops byte offset or -1, tc_bias index or -1, 0) for MLP value i
cudaError_t launch_derive(const float* planes, long long n_planes, __nv_bfloat16* planes_bf16, const float* mlp,
                          int n_mlp, const int4* tab, float* mlp_t, uint8_t* tc_ops, float* tc_bias, cudaStream_t s);
}  // namespace fs4d

// ================================================================ backward
namespace fs4d {

constexpr int kPairGrad = 9;  // per (tile, Gaussian) pair: du dv dconic(a b c) dopacity drgb(3)
constexpr int kPairStride = 12;  // floats per pair slot in memory (16-byte aligned rows)

struct CompositeBwdArgs {
  int width, height, tiles_x;
  const uint2* ranges;
  const uint32_t* values;
  const float2* xy;
  const float4* conic_opacity;
  const float* rgb;
  const int4* rect;
  const uint32_t* offsets;
  const float* t_final;
  const int* n_contrib;
  const float* dl_dimage;   // [H][W][3]
  float* grad_pair;         // [K][kPairStride] (9 used), indexed by emission slot; zeroed by the caller
};

struct ProjectBwdArgs {
  int n;
  const float* means;       // deformed [n][3]
  const float* quats;       // deformed [n][4]
  const float* log_scales;  // deformed [n][3]
  const float* sh;          // [n][K][3]
  int sh_degree;
  CamParams cam;
  const float4* conic_opacity;
  const int* radius;
  const int4* rect;
  const uint32_t* offsets;
  const float* grad_pair;
  float* gd;                // out [n][10]: dL/d(X', r', s')
  float* g_means;           // += (nullable)
  float* g_quats;
  float* g_log_scales;
  float* g_opacity;
  float* g_sh;
  float* stat_grad;         // += |dL/d(projected mean)| where visible (nullable)
  float* stat_visible;      // += 1 where visible (nullable)
};

// Per-Gaussian activations and deltas of the deformation MLP, feature-major
// ([feature][n]) so that each thread's writes coalesce across the warp.
struct MlpActs {
  float* fh;    // [HL][n]  layer d1 input
  float* a1;    // [64][n]  layer d2 input
  float* fd;    // [64][n]  head hidden-layer input
  float* hid;   // [192][n] head output-layer inputs (x, r, s)
  float* dout;  // [10][n]  output deltas
  float* dh;    // [192][n] head hidden pre-activation deltas
  float* d2;    // [64][n]
  float* d1;    // [64][n]
};

struct MlpBwdArgs {
  DeformArgs f;             // canonical scene, t0, planes, transposed MLP
  const float* gd;          // [n][10]
  MlpActs act;
  float* g_planes;          // += (nullable)
  float* g_means;           // += (nullable)
};

cudaError_t launch_composite_bwd(const CompositeBwdArgs& a, cudaStream_t s);
cudaError_t launch_project_bwd(const ProjectBwdArgs& a, cudaStream_t s);
cudaError_t launch_mlp_bwd(const MlpBwdArgs& a, cudaStream_t s);
// dW[o][i] += sum_n D[o][n] X[i][n], db[o] += sum_n D[o][n] for up to 8 layers in one launch, through
// per-chunk partial sums (deterministic two-stage reduction).  W and b in the source layout
// (W[out][in] then b); D [O][n], X [I][n] feature-major.
struct WgradLayer {
  const float* D;
  const float* X;
  int O, I;
  float* gW;
  float* gb;
  long long part_off;  // set by launch_wgrad
};
struct WgradArgs {
  WgradLayer l[8];
  int n_layers;
  long long n;
  int chunks;          // set by launch_wgrad
  float* partial;      // wgrad_chunks(n) x sum of (O*I + O) floats
};
long long wgrad_chunks(long long n);
cudaError_t launch_wgrad(WgradArgs& a, cudaStream_t s);

// Densification and pruning (densify.cu).
struct DensifyArgs {
  int n;
  const float* log_scales;  // [n][3]
  const float* opacity;     // [n] logits
  const float* grad_sum;    // [n]
  const float* visible;     // [n]
  float grad_threshold, split_log_scale, prune_logit;
  uint32_t* block_off;      // [3][densify_blocks(n)]: per-block counts, then their exclusive prefixes
  uint32_t* totals;         // [3]: kept, copied, split
  int32_t* src;             // [n_out] (map): source Gaussian of each output
  int32_t* kind;            // [n_out] (map): 0 kept, 1 copy, 2 first child, 3 second child
};
struct ChildArgs {
  long long first, end;     // the children's output range
  const int32_t* src;
  const int32_t* kind;
  const float* means;       // old [n][3]
  const float* log_scales;  // old [n][3]
  const float* quats;       // old [n][4]
  const float* normals;     // [n][2][3]
  float* out_means;         // new [n_out][3]
  float* out_log_scales;    // new [n_out][3]
};
int densify_blocks(int n);
cudaError_t launch_densify_plan(const DensifyArgs& a, cudaStream_t s);
cudaError_t launch_densify_map(const DensifyArgs& a, cudaStream_t s);
cudaError_t launch_gather(const float* in, float* out, const int32_t* src, const int32_t* kind, long long n_out,
                          int width, bool zero_new, cudaStream_t s);
cudaError_t launch_children(const ChildArgs& a, cudaStream_t s);
cudaError_t launch_morton(const float* means, int n, const float lo[3], const float hi[3], unsigned long long* keys,
                          uint32_t* values, cudaStream_t s);

}  // namespace fs4d

namespace fs4d {
// Gaussian weight of Eq. 1 as a power of two: with the conic (a, b, c) scaled
// once per Gaussian by log2(e) into (a2, b2, c2) = log2(e) * (-a/2, -b, -c/2),
// exp(-d^T K d / 2) = 2^(a2 dx^2 + b2 dx dy + c2 dy^2), one SFU instruction.
// Forward and backward compositing share this exact arithmetic, so the backward
// reproduces every forward decision bit for bit.
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float ex2_approx(float y) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
  return r;
}

__device__ __forceinline__ float4 composite_coeffs(float2 p, float4 conic_opacity) {
  return make_float4(p.x, p.y, (-0.5f * kLog2e) * conic_opacity.x, (-0.5f * kLog2e) * conic_opacity.z);
}
__device__ __forceinline__ float composite_b2(float4 conic_opacity) { return -kLog2e * conic_opacity.y; }

// alpha = min(0.99, o * G) of a term at offset (dx, dy) = mean - pixel centre,
// or 0 when the term is skipped (alpha below 1/255).  The exponent
// dx (a2 dx + b2 dy) + c2 dy^2 is never positive: every Gaussian that reaches
// compositing has a positive-definite conic (projection culls det <= 0, and the
// 0.3 dilation keeps det >= 0.09), so no exponent-sign test is needed.
__device__ __forceinline__ float composite_alpha(const float4& g0, float b2, float opacity, float dx, float dy,
                                                 float& G) {
  const float p = fmaf(fmaf(g0.z, dx, b2 * dy), dx, (g0.w * dy) * dy);
  G = ex2_approx(p);
  const float alpha = fminf(0.99f, opacity * G);
  return alpha < 1.f / 255.f ? 0.f : alpha;
}

// Minimum over t in [t0, t1] of A u^2 + 2 B u t + C t^2 for fixed u (C > 0), whose
// unconstrained minimiser is t = k u with k = -B / C.
__device__ __forceinline__ float edge_min(float A, float B, float C, float k, float u, float t0, float t1) {
  const float t = fminf(t1, fmaxf(t0, k * u));
  return A * u * u + 2.f * B * u * t + C * t * t;
}

// Minimum of the positive-definite quadratic q(x, y) = A x^2 + 2 B x y + C y^2 over
// the rectangle [x0, x1] x [y0, y1] (coordinates relative to the mean): 0 if the
// mean lies inside, else the least of the four edges' minima (each in closed form;
// a rounded minimiser only raises q by a second-order amount).  kx = -B / C,
// ky = -B / A.
__device__ __forceinline__ float rect_min(float A, float B, float C, float kx, float ky, float x0, float x1,
                                          float y0, float y1) {
  if (x0 <= 0.f && x1 >= 0.f && y0 <= 0.f && y1 >= 0.f) return 0.f;
  return fminf(fminf(edge_min(A, B, C, kx, x0, y0, y1), edge_min(A, B, C, kx, x1, y0, y1)),
               fminf(edge_min(C, B, A, ky, y0, x0, x1), edge_min(C, B, A, ky, y1, x0, x1)));
}

// Natural-log exponent bound: a term reaches alpha >= 1/255 only where
// -d^T K d / 2 >= ln(1/(255 o)); the bound minus 1e-3 (0.1% in alpha, far above
// the rounding of either exponent form) is used for conservative culling.
__device__ __forceinline__ float composite_exp_threshold(float opacity) {
  return logf((1.f / 255.f) / opacity) - 1e-3f;
}
}  // namespace fs4d
