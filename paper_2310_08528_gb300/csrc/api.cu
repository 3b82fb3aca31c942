// C ABI of libfs4d.so: contexts, resident scenes, work memory and the per-frame
// launch sequence: deform -> project -> depth sort of the N Gaussians -> tile
// binning (tile bitmap: mark -> tile scan -> extract; or key emission -> tile
// scan -> stable pair sort on the tile bits) -> composite.  See include/fs4d.h
// for the contract of every call.
#include <nvtx3/nvToolsExt.h>
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "fs4d_internal.cuh"

namespace fs4d {
thread_local unsigned long long g_kernel_launches = 0;
}  // namespace fs4d

using namespace fs4d;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

#ifdef FS4D_CHECK_BOUNDS
// Debug build: canary bytes after every buffer, and the registry of live buffers.
constexpr size_t kCanaryBytes = 256;
constexpr unsigned char kCanary = 0xA5;
std::mutex g_canary_mu;
std::map<void*, size_t> g_canaries;  // buffer -> its size (the canary follows)
void* g_last_buffer = nullptr;
#else
constexpr size_t kCanaryBytes = 0;
#endif

cudaError_t ensure(DevBuf& b, size_t bytes);
void release(DevBuf& b) {
#ifdef FS4D_CHECK_BOUNDS
  if (b.p) {
    std::lock_guard<std::mutex> lock(g_canary_mu);
    g_canaries.erase(b.p);
    if (g_last_buffer == b.p) g_last_buffer = nullptr;
  }
#endif
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

cudaError_t ensure(DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return cudaSuccess;
  if (b.p) {
#ifdef FS4D_CHECK_BOUNDS
    {
      std::lock_guard<std::mutex> lock(g_canary_mu);
      g_canaries.erase(b.p);
      if (g_last_buffer == b.p) g_last_buffer = nullptr;
    }
#endif
    cudaError_t e = cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (e != cudaSuccess) return e;
  }
  if (bytes == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(&b.p, bytes + kCanaryBytes);
  if (e == cudaSuccess) b.bytes = bytes;
#ifdef FS4D_CHECK_BOUNDS
  if (e == cudaSuccess) {
    e = cudaMemset(static_cast<unsigned char*>(b.p) + bytes, kCanary, kCanaryBytes);
    std::lock_guard<std::mutex> lock(g_canary_mu);
    g_canaries[b.p] = bytes;
    g_last_buffer = b.p;
  }
#endif
  return e;
}

template <typename T>
T* P(DevBuf& b) {
  return reinterpret_cast<T*>(b.p);
}

struct Scene {
  int id = 0;
  fs4d_scene_desc shape{};  // the load call's sizes and box (its pointers cleared)
  int n = 0, sh_degree = 0, K = 1;
  DevBuf means, log_scales, quats, opacity_logits, sh;
  DevBuf planes, planes_bf16, mlp, mlp_t, tc_ops, tc_bias;
  DevBuf derive_tab;  // per MLP value: its places in mlp_t, tc_ops and tc_bias (device-side refresh)
  DevBuf perm;  // deformation work order: Gaussians by Morton code of their canonical mean
  PlaneGeom pg{};
  MlpGeomT mg{};
  MlpGeomTC tg{};
  size_t planes_floats = 0, mlp_floats = 0;
  size_t resident = 0;
  bool bf16_ok = false;
  bool color_heads = false;   // App. B colour and opacity heads, at float offset color_off of mlp
  size_t color_off = 0;
  std::atomic<int> refs{0};   // serving requests in flight on this scene
  bool dying = false;         // being unloaded: no new serving launches
  // capacity-mode reservation
  long long reserved_pairs = 0;
  int reserved_w = 0, reserved_h = 0;
};

// Per-context work memory, grown on demand (never during a capture).
// Per-frame state that must start at zero (histograms, tickets, selection words,
// pair count, tile counts, look-back tables), carved out of one allocation that
// ONE memset clears at the start of a frame.
struct FrameZero {
  uint32_t* hist = nullptr;              // [8][256]: depth-key byte histograms, then the pair sort's
  uint32_t* counters = nullptr;          // [64]: [0] emission ticket, [8, 25) depth sort, [32, 49) pair sort
  uint32_t* num_pairs = nullptr;         // [4]
  uint32_t* tile_count = nullptr;        // [n_tiles]
  unsigned long long* emit_lb = nullptr; // [emit_parts(n) + 1]
  uint32_t* dlb = nullptr;               // depth-sort look-back [4][dparts][256]
  uint32_t* plb = nullptr;               // pair-sort look-back [passes][pparts][256]
  long long dparts = 0, pparts = 0;
  size_t bytes = 0;
};

struct Work {
  DevBuf zero;                             // FrameZero's allocation
  FrameZero z;                             // its layout for the frame in flight
  DevBuf dmeans, dquats, dscales;          // deformed Gaussians
  DevBuf xy, co, rgb, depth, radius, rect; // projected
  DevBuf offsets, emit_lb, counters, num_pairs, hist;
  DevBuf dkeys, dvals, dkeys_alt, dvals_alt;  // per-Gaussian depth sort
  DevBuf keys, values, keys_alt, values_alt;
  DevBuf sort_lb;
  DevBuf ranges, tile_count, tile_order;
  DevBuf bitmap;                           // tile bitmap binning: [tiles][bitmap_words(n)], zero between frames
  DevBuf sxy, sco, srgb;                   // with the bitmap: projected Gaussians in depth-rank order
  bool bmp = false;                        // the frame in flight bins through the bitmap
  bool packed = false;                     // ... or sorts (tile | index) keys without values
  bool bmp_dirty = false;                  // a frame set bits whose extraction was not launched
  DevBuf ts;
  DevBuf host_img;                         // device staging image of fs4d_render_host
  DevBuf grad_pair, gd, acts, wpartial;    // backward work memory
  DevBuf fd, dsh, dop;                     // colour and opacity heads: f_d [n][64] (work order),
                                           // deformed SH [n][48] and opacity logits [n]
  int cap_color = 0;
  long long cap_pairs = 0;
  long long sort_parts_cap = 0;
  int cap_n = 0, cap_tiles = 0;
};

constexpr int kSortMaxPasses = 8;
// Largest tile bitmap (one bit per (tile, Gaussian)) a frame bins through; larger
// frames emit keys and radix-sort them.  At this size clearing and walking the
// rows costs about as much memory traffic as the sort's passes over ~10 pairs per
// Gaussian, and the sort's latency chains are gone.
constexpr size_t kBitmapMaxBytes = size_t(256) << 20;

size_t bitmap_bytes(int n, long long n_tiles) { return 4 * (size_t)n_tiles * (size_t)bitmap_words(std::max(n, 1)); }
constexpr int kCounters = 32;  // [0] emit ticket, [8, 25) radix-sort tickets and selection words
constexpr int kEmitCounters = 8;  // the words reset before an emission (the sort's words stay)

// Byte layout of FrameZero for n Gaussians, n_tiles tiles, cap pairs and a pair
// sort of pair_passes passes (256-byte aligned blocks); fills z when base != NULL.
size_t frame_zero_layout(int n, int n_tiles, long long cap, int pair_passes, unsigned char* base, FrameZero* z) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  const long long dparts = sort_parts(std::max(n, 1)), pparts = sort_parts(std::max<long long>(cap, 1));
  const size_t o_hist = take(4 * 256 * (size_t)kSortMaxPasses);
  const size_t o_cnt = take(4 * 64);
  const size_t o_np = take(16);
  const size_t o_tc = take(4 * (size_t)n_tiles);
  const size_t o_elb = take(8 * (size_t)(emit_parts(std::max(n, 1)) + 1));
  const size_t o_dlb = take(4 * 256 * 4 * (size_t)dparts);
  const size_t o_plb = take(4 * 256 * (size_t)pair_passes * pparts);
  if (base && z) {
    z->hist = reinterpret_cast<uint32_t*>(base + o_hist);
    z->counters = reinterpret_cast<uint32_t*>(base + o_cnt);
    z->num_pairs = reinterpret_cast<uint32_t*>(base + o_np);
    z->tile_count = reinterpret_cast<uint32_t*>(base + o_tc);
    z->emit_lb = reinterpret_cast<unsigned long long*>(base + o_elb);
    z->dlb = reinterpret_cast<uint32_t*>(base + o_dlb);
    z->plb = reinterpret_cast<uint32_t*>(base + o_plb);
    z->dparts = dparts;
    z->pparts = pparts;
    z->bytes = off;
  }
  return off;
}

}  // namespace

// Forward state of one rendered frame, owned by the frame (device copies), so
// that the context's work memory can be reused before the backward runs.
struct fs4d_frame {
  int scene = -1;
  fs4d_camera cam{};
  float t = 0.f;
  int n = 0;
  long long pairs = 0;
  DevBuf dmeans, dquats, dscales;              // deformed Gaussians
  DevBuf xy, co, rgb, radius, rect, offsets;   // projection and emission offsets
  DevBuf values, ranges;                       // sorted Gaussian indices, per-tile ranges
  DevBuf t_final, n_contrib;                   // per pixel
};

struct fs4d_server;

struct fs4d_ctx {
  std::mutex mu;                 // guards the scene map (the serving thread reads it)
  fs4d_server* server = nullptr;
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  std::map<int, Scene*> scenes;
  int next_id = 1;
  Work w;
  DevBuf status;
  uint32_t* h_pinned = nullptr;  // [4] readback slots
  long long last_pairs = 0;
  uint32_t* last_values = nullptr;  // sorted Gaussian indices of the last frame (work memory)
  int binning = FS4D_BINNING_AUTO;
  int last_binning = FS4D_BINNING_SORT;
  bool timing = false;
  cudaEvent_t ev[8] = {};        // start, deformed, projected, depth-sorted, binned | pair sort, sorted, composited
  cudaEvent_t bev[5] = {};       // backward: start, compositing, projection, MLP + planes, weight gradients done
  // fs4d_render_host_batch: image copies overlapped with the next frame
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t slot_rendered[2] = {}, slot_copied[2] = {};
  unsigned long long* h_pairs = nullptr;  // pinned, [h_pairs_cap]: each frame's pair count
  int h_pairs_cap = 0;
  uint32_t spin_limit = kSpinLimit;       // polls of a look-back wait (fs4d_set_wait_limit)
  // frames rendered in bands of tile rows (more pairs than one sort pass counts)
  int band_scene = -1, band_w = 0, band_h = 0, band_hint = 0;  // bands the last such frame used
  std::vector<std::pair<int, int>> band_rows;  // ... and their tile rows (the next frame reuses them)
  int last_bands = 1;
  long long last_launches = 0;  // kernels the last fs4d_render / fs4d_render_async call launched
  long long band_pairs = (1ll << 30) - 1;  // most pairs one band may hold (fs4d_set_band_pairs)
  float stage_acc[6] = {};                // stage times summed over a banded frame's passes
  bool stage_acc_valid = false;
};

namespace {

fs4d_status fail(fs4d_ctx* c, fs4d_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

fs4d_status cuda_fail(fs4d_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(c, e == cudaErrorMemoryAllocation ? FS4D_ERR_OOM : FS4D_ERR_CUDA, m);
}

#define FS4D_CUDA(ctx, expr)                                   \
  do {                                                         \
    cudaError_t e_ = (expr);                                   \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #expr); \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Record stage event i (as an external event node when the stream is being
// captured, so that replays of the graph still time the stage).
void mark(fs4d_ctx* c, int i) {
  if (!c->timing) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(c->stream, &cs);
  if (cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(c->ev[i], c->stream, cudaEventRecordExternal);
  else
    cudaEventRecord(c->ev[i], c->stream);
}

int ceil_log2(long long v) {
  int b = 0;
  while ((1ll << b) < v) ++b;
  return b;
}

int tiles_of(int px) { return (px + kTile - 1) / kTile; }

CamParams cam_params(const fs4d_camera& c) {
  CamParams p;
  p.width = c.width; p.height = c.height;
  p.fx = c.fx; p.fy = c.fy; p.cx = c.cx; p.cy = c.cy; p.znear = c.znear;
  for (int i = 0; i < 12; ++i) p.m[i] = c.world_to_cam[i];
  p.guard_w = c.width; p.guard_h = c.height;
  return p;
}

bool valid_cam(const fs4d_camera* c) {
  return c && c->width > 0 && c->height > 0 && c->width <= 8192 && c->height <= 8192 && c->fx > 0 && c->fy > 0;
}

// Plane geometry: level-major, then xy xz yz xt yt zt; [R_b][R_a][h] each.
void plane_geom(const fs4d_scene_desc& d, PlaneGeom& pg, size_t& total) {
  static const int ax[6] = {0, 0, 1, 0, 1, 2}, bx[6] = {1, 2, 2, 3, 3, 3};
  pg.n_levels = d.n_levels;
  pg.feat_dim = d.feat_dim;
  pg.res_time = d.res_time;
  long long off = 0;
  for (int l = 0; l < kMaxLevels; ++l) {
    pg.res[l] = l < d.n_levels ? d.res_spatial[l] : 0;
    for (int p = 0; p < 6; ++p) {
      pg.off[l][p] = off;
      if (l < d.n_levels) {
        const long long Ra = ax[p] < 3 ? d.res_spatial[l] : d.res_time;
        const long long Rb = bx[p] < 3 ? d.res_spatial[l] : d.res_time;
        off += Ra * Rb * d.feat_dim;
      }
    }
  }
  for (int a = 0; a < 3; ++a) {
    pg.aabb_min[a] = d.aabb_min[a];
    pg.aabb_scale[a] = 2.f / (d.aabb_max[a] - d.aabb_min[a]);
  }
  total = (size_t)off;
}

// Offsets of the source MLP layout (W[out][in] then b[out], d1 d2 x1 x2 r1 r2 s1 s2).
struct SrcLayer {
  int out, in;
  size_t w, b;
};

std::vector<SrcLayer> src_layers(int hin, int W, size_t* total) {
  const int outs[8] = {W, W, W, 3, W, 4, W, 3};
  const int ins[8] = {hin, W, W, W, W, W, W, W};
  std::vector<SrcLayer> L(8);
  size_t off = 0;
  for (int k = 0; k < 8; ++k) {
    L[k].out = outs[k]; L[k].in = ins[k];
    L[k].w = off; off += (size_t)outs[k] * ins[k];
    L[k].b = off; off += outs[k];
  }
  *total = off;
  return L;
}

// Floats of a scene's MLP array: the eight layers, and the colour and opacity heads.
size_t mlp_floats_of(const fs4d_scene_desc& d) {
  size_t total = 0;
  src_layers(d.feat_dim * d.n_levels, d.mlp_width, &total);
  if (d.color_heads) total += (size_t)color_layer_floats(3 * (d.sh_degree + 1) * (d.sh_degree + 1));
  return total;
}

// FP32 kernel layout: every layer transposed, Wt[in][out] then b[out], each
// block padded to a multiple of 4 floats.
std::vector<float> transpose_mlp(const float* src, int hin, int W, MlpGeomT& mg) {
  size_t tot;
  auto L = src_layers(hin, W, &tot);
  std::vector<float> out;
  mg.hin = hin;
  auto pad = [&]() { while (out.size() % 4) out.push_back(0.f); };
  for (int k = 0; k < 8; ++k) {
    pad();
    mg.w[k] = (int)out.size();
    for (int i = 0; i < L[k].in; ++i)
      for (int o = 0; o < L[k].out; ++o) out.push_back(src[L[k].w + (size_t)o * L[k].in + i]);
    pad();
    mg.b[k] = (int)out.size();
    for (int o = 0; o < L[k].out; ++o) out.push_back(src[L[k].b + o]);
  }
  pad();
  mg.total = (int)out.size();
  return out;
}

uint16_t f2bf(float f) {  // round to nearest even
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}

// Byte offset of element (row r, k) of a K-major operand in the canonical
// no-swizzle layout: 8-row x 16-byte core matrices, core (r/8, k/8) at
// ((r/8) * (K/8) + k/8) * 128 bytes, element at (r%8)*16 + (k%8)*2 inside.
size_t umma_off(int r, int k, int Kdim) {
  return ((size_t)(r / 8) * (Kdim / 8) + (k / 8)) * 128 + (r % 8) * 16 + (k % 8) * 2;
}

// BF16 tensor-core operand image: B1 = d1 [64 x hin], B2 = d2 [64 x 64],
// B3 = [x1; r1; s1] [192 x 64], B4 = block-diag(x2, r2, s2) padded [16 x 192].
void build_tc_image(const float* src, int hin, int W, MlpGeomTC& tg, std::vector<uint8_t>& img,
                    std::vector<float>& bias) {
  size_t tot;
  auto L = src_layers(hin, W, &tot);
  tg.hin = hin;
  tg.b1_off = 0;
  tg.b2_off = tg.b1_off + 64 * hin * 2;
  tg.b3_off = tg.b2_off + 64 * 64 * 2;
  tg.b4_off = tg.b3_off + 192 * 64 * 2;
  tg.bytes = tg.b4_off + 16 * 192 * 2;
  img.assign(tg.bytes, 0);
  auto put = [&](int base, int r, int k, int Kdim, float v) {
    const uint16_t b = f2bf(v);
    std::memcpy(&img[base + umma_off(r, k, Kdim)], &b, 2);
  };
  for (int o = 0; o < 64; ++o)
    for (int i = 0; i < hin; ++i) put(tg.b1_off, o, i, hin, src[L[0].w + (size_t)o * hin + i]);
  for (int o = 0; o < 64; ++o)
    for (int i = 0; i < 64; ++i) put(tg.b2_off, o, i, 64, src[L[1].w + (size_t)o * 64 + i]);
  for (int h = 0; h < 3; ++h)
    for (int o = 0; o < 64; ++o)
      for (int i = 0; i < 64; ++i) put(tg.b3_off, 64 * h + o, i, 64, src[L[2 + 2 * h].w + (size_t)o * 64 + i]);
  const int col0[3] = {0, 3, 7};
  for (int h = 0; h < 3; ++h)
    for (int j = 0; j < L[3 + 2 * h].out; ++j)
      for (int i = 0; i < 64; ++i) put(tg.b4_off, col0[h] + j, 64 * h + i, 192, src[L[3 + 2 * h].w + (size_t)j * 64 + i]);
  bias.assign(64 + 64 + 192 + 16, 0.f);
  tg.bias_off[0] = 0; tg.bias_off[1] = 64; tg.bias_off[2] = 128; tg.bias_off[3] = 320;
  tg.bias_total = 336;
  for (int o = 0; o < 64; ++o) bias[o] = src[L[0].b + o];
  for (int o = 0; o < 64; ++o) bias[64 + o] = src[L[1].b + o];
  for (int h = 0; h < 3; ++h)
    for (int o = 0; o < 64; ++o) bias[128 + 64 * h + o] = src[L[2 + 2 * h].b + o];
  for (int h = 0; h < 3; ++h)
    for (int j = 0; j < L[3 + 2 * h].out; ++j) bias[320 + col0[h] + j] = src[L[3 + 2 * h].b + j];
}

// For every value of the source-layout MLP, where transpose_mlp and
// build_tc_image put it: (mlp_t index, tc_ops byte offset or -1, tc_bias index or
// -1, 0).  Lets a kernel refresh both derived layouts after the MLP changes on
// the device.
std::vector<int4> build_derive_tab(int hin, int W, const MlpGeomT& mg, const MlpGeomTC& tg, bool with_tc) {
  size_t tot;
  auto L = src_layers(hin, W, &tot);
  std::vector<int4> tab(tot, make_int4(0, -1, -1, 0));
  const int col0[3] = {0, 3, 7};
  for (int k = 0; k < 8; ++k) {
    for (int o = 0; o < L[k].out; ++o) {
      for (int i = 0; i < L[k].in; ++i) tab[L[k].w + (size_t)o * L[k].in + i].x = mg.w[k] + i * L[k].out + o;
      tab[L[k].b + o].x = mg.b[k] + o;
    }
    if (!with_tc) continue;
    const int h = (k - 2) / 2;  // head of layers 2..7
    for (int o = 0; o < L[k].out; ++o) {
      int4& b = tab[L[k].b + o];
      b.z = k == 0 ? o : k == 1 ? 64 + o : (k % 2 == 0) ? 128 + 64 * h + o : 320 + col0[h] + o;
      for (int i = 0; i < L[k].in; ++i) {
        int4& e = tab[L[k].w + (size_t)o * L[k].in + i];
        if (k == 0) e.y = tg.b1_off + (int)umma_off(o, i, hin);
        else if (k == 1) e.y = tg.b2_off + (int)umma_off(o, i, 64);
        else if (k % 2 == 0) e.y = tg.b3_off + (int)umma_off(64 * h + o, i, 64);
        else e.y = tg.b4_off + (int)umma_off(col0[h] + o, 64 * h + i, 192);
      }
    }
  }
  return tab;
}

template <typename T>
fs4d_status upload(fs4d_ctx* c, DevBuf& b, const T* h, size_t count, size_t* acc) {
  FS4D_CUDA(c, ensure(b, sizeof(T) * std::max<size_t>(count, 1)));
  if (count) FS4D_CUDA(c, cudaMemcpy(b.p, h, sizeof(T) * count, cudaMemcpyHostToDevice));
  *acc += b.bytes;
  return FS4D_OK;
}

void free_scene(Scene* s) {
  DevBuf* all[] = {&s->means, &s->log_scales, &s->quats, &s->opacity_logits, &s->sh, &s->planes,
                   &s->planes_bf16, &s->mlp, &s->mlp_t, &s->tc_ops, &s->tc_bias, &s->perm, &s->derive_tab};
  for (DevBuf* b : all) release(*b);
  delete s;
}

fs4d_status get_scene(fs4d_ctx* c, fs4d_scene_id id, Scene** out) {
  std::lock_guard<std::mutex> lock(c->mu);
  auto it = c->scenes.find(id);
  if (it == c->scenes.end() || it->second->dying)
    return fail(c, FS4D_ERR_NOT_FOUND, "unknown scene id " + std::to_string(id));
  *out = it->second;
  return FS4D_OK;
}

// Grow the per-Gaussian / per-tile / per-pair work buffers.
// Work memory of the colour and opacity heads for frames of up to n Gaussians
// (allocated on the first frame of a scene with them; never during a capture).
fs4d_status ensure_color(fs4d_ctx* c, Work& w, cudaStream_t stream, int n) {
  if (w.cap_color >= n) return FS4D_OK;
  FS4D_CUDA(c, cudaStreamSynchronize(stream));
  FS4D_CUDA(c, ensure(w.fd, 4 * 64 * (size_t)n + 16384));  // + the last BF16 tile image's ragged end
  FS4D_CUDA(c, ensure(w.dsh, 4 * 48 * (size_t)n));
  FS4D_CUDA(c, ensure(w.dop, 4 * (size_t)n));
  w.cap_color = n;
  return FS4D_OK;
}

fs4d_status ensure_work(fs4d_ctx* c, Work& w, cudaStream_t stream, int n, int n_tiles, long long pairs) {
  const bool bmp_ok = c->binning != FS4D_BINNING_SORT;
  const size_t bmp_need =
      std::max(bitmap_bytes(std::max(n, w.cap_n), std::max(n_tiles, w.cap_tiles)), w.bitmap.bytes);
  const bool bmp_grow = bmp_ok && bmp_need <= kBitmapMaxBytes && bmp_need > w.bitmap.bytes;
  bool grow = n > w.cap_n || n_tiles > w.cap_tiles || pairs > w.cap_pairs || bmp_grow;
  if (!grow) return FS4D_OK;
  FS4D_CUDA(c, cudaStreamSynchronize(stream));
  if (n > w.cap_n) {
    const size_t m = (size_t)n;
    FS4D_CUDA(c, ensure(w.dmeans, 12 * m));
    FS4D_CUDA(c, ensure(w.dquats, 16 * m));
    FS4D_CUDA(c, ensure(w.dscales, 12 * m));
    FS4D_CUDA(c, ensure(w.xy, 8 * m));
    FS4D_CUDA(c, ensure(w.co, 16 * m));
    FS4D_CUDA(c, ensure(w.rgb, 12 * m));
    FS4D_CUDA(c, ensure(w.depth, 4 * m));
    FS4D_CUDA(c, ensure(w.radius, 4 * m));
    FS4D_CUDA(c, ensure(w.rect, 16 * m));
    FS4D_CUDA(c, ensure(w.sxy, 8 * m));
    FS4D_CUDA(c, ensure(w.sco, 16 * m));
    FS4D_CUDA(c, ensure(w.srgb, 12 * m));
    FS4D_CUDA(c, ensure(w.offsets, 4 * m));
    FS4D_CUDA(c, ensure(w.emit_lb, 8 * (size_t)(emit_parts(n) + 1)));
    FS4D_CUDA(c, ensure(w.dkeys, 8 * m));
    FS4D_CUDA(c, ensure(w.dvals, 4 * m));
    FS4D_CUDA(c, ensure(w.dkeys_alt, 8 * m));
    FS4D_CUDA(c, ensure(w.dvals_alt, 4 * m));
    w.cap_n = n;
  }
  FS4D_CUDA(c, ensure(w.counters, 4 * kCounters));
  FS4D_CUDA(c, ensure(w.num_pairs, 4 * 4));
  FS4D_CUDA(c, ensure(w.hist, 4 * 256 * kSortMaxPasses));
  if (n_tiles > w.cap_tiles) {
    FS4D_CUDA(c, ensure(w.ranges, 8 * (size_t)n_tiles));
    FS4D_CUDA(c, ensure(w.tile_count, 4 * (size_t)n_tiles));
    FS4D_CUDA(c, ensure(w.tile_order, 4 * (size_t)n_tiles));
    w.cap_tiles = n_tiles;
  }
  if (pairs > w.cap_pairs) {
    const long long cap = std::max<long long>(pairs, 4096);
    FS4D_CUDA(c, ensure(w.keys, 8 * (size_t)cap));
    FS4D_CUDA(c, ensure(w.values, 4 * (size_t)cap));
    FS4D_CUDA(c, ensure(w.keys_alt, 8 * (size_t)cap));
    FS4D_CUDA(c, ensure(w.values_alt, 4 * (size_t)cap));
    w.cap_pairs = cap;
  }
  const long long parts = std::max(sort_parts(std::max<long long>(w.cap_pairs, 4096)), sort_parts(w.cap_n));
  if (parts > w.sort_parts_cap) {
    FS4D_CUDA(c, ensure(w.sort_lb, 4 * 256 * (size_t)kSortMaxPasses * parts));
    w.sort_parts_cap = parts;
  }
  const size_t zb = frame_zero_layout(w.cap_n, w.cap_tiles, w.cap_pairs,
                                      sort_passes(ceil_log2(std::max(w.cap_tiles, 1))), nullptr, nullptr);
  FS4D_CUDA(c, ensure(w.zero, zb));
  if (bmp_grow) {  // zeroed once here; every frame that sets bits clears them again
    FS4D_CUDA(c, ensure(w.bitmap, bmp_need));
    FS4D_CUDA(c, cudaMemsetAsync(w.bitmap.p, 0, w.bitmap.bytes, stream));
    w.bmp_dirty = false;
    FS4D_CUDA(c, cudaStreamSynchronize(stream));
  }
  return FS4D_OK;
}

// Whether a frame of n Gaussians over n_tiles tiles bins through w's bitmap.
bool use_bitmap(const fs4d_ctx* c, const Work& w, int n, int n_tiles, bool offsets) {
  const size_t b = bitmap_bytes(n, n_tiles);
  return c->binning != FS4D_BINNING_SORT && !offsets && n > 0 && b <= kBitmapMaxBytes && b <= w.bitmap.bytes;
}

fs4d_status ensure_work(fs4d_ctx* c, int n, int n_tiles, long long pairs) {
  return ensure_work(c, c->w, c->stream, n, n_tiles, pairs);
}

SortWork sort_work(Work& w) {
  SortWork sw;
  sw.hist = P<uint32_t>(w.hist);
  sw.lookback = P<uint32_t>(w.sort_lb);
  sw.part_counters = P<uint32_t>(w.counters) + 8;
  sw.max_parts = w.sort_parts_cap;
  return sw;
}

SortWork sort_work(fs4d_ctx* c) {
  SortWork sw = sort_work(c->w);
  sw.spin_limit = c->spin_limit;
  return sw;
}

// Where one frame's launches go: work memory, stream, status word, and whether
// the context's stage-timing events are recorded.
struct Env {
  fs4d_ctx* c;
  Work* w;
  cudaStream_t s;
  uint32_t* status;
  bool timed;
  int guard_w = 0, guard_h = 0;  // non-zero: the whole frame's size (a band's guard band is the frame's)
};

Env env_of(fs4d_ctx* c) { return Env{c, &c->w, c->stream, P<uint32_t>(c->status), true}; }

// Stage boundaries of a frame (0 start, 1 deformed, 2 projected, 3 depth-sorted,
// 4 binned, 5 pair sort start, 6 pair-sorted, 7 composited): CUDA events when stage
// timing is on, and NVTX ranges named after the stages for profilers (a no-op
// unless a tool is attached).
void mark(const Env& e, int i) {
  static const char* const kRange[8] = {"fs4d:deform", "fs4d:project", "fs4d:depth_sort", "fs4d:binning", nullptr,
                                        "fs4d:pair_sort", "fs4d:composite", nullptr};
  if (i != 0 && i != 5) nvtxRangePop();
  if (kRange[i]) nvtxRangePushA(kRange[i]);
  if (e.timed) mark(e.c, i);
}

// An NVTX range over one call of the library.
struct NvtxScope {
  explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
  ~NvtxScope() { nvtxRangePop(); }
};

DeformArgs deform_args(Scene* s, const float* ts, float t0, int n_t, float* om, float* oq, float* os) {
  DeformArgs a{};
  a.n = s->n; a.n_t = n_t; a.ts = ts; a.t0 = t0;
  a.perm = P<uint32_t>(s->perm);
  a.means = P<float>(s->means); a.quats = P<float>(s->quats); a.log_scales = P<float>(s->log_scales);
  a.out_means = om; a.out_quats = oq; a.out_log_scales = os;
  a.planes = P<float>(s->planes);
  a.planes_bf16 = P<__nv_bfloat16>(s->planes_bf16);
  a.mlp_t = P<float>(s->mlp_t);
  a.mg = s->mg;
  a.tc_ops = P<uint8_t>(s->tc_ops);
  a.tc_bias = P<float>(s->tc_bias);
  a.tg = s->tg;
  a.pg = s->pg;
  return a;
}

fs4d_status run_deform(fs4d_ctx* c, Scene* s, fs4d_precision prec, const DeformArgs& a, cudaStream_t stream,
                       uint32_t* status) {
  DeformArgs b = a;
  b.status = status;
  if (prec == FS4D_BF16) {
    if (!s->bf16_ok) return fail(c, FS4D_ERR_UNIMPLEMENTED, "BF16 deformation does not support this scene shape");
    FS4D_CUDA(c, launch_deform_bf16(b, stream));
  } else {
    FS4D_CUDA(c, launch_deform_fp32(b, stream));
  }
  return FS4D_OK;
}

fs4d_status run_deform(fs4d_ctx* c, Scene* s, fs4d_precision prec, const DeformArgs& a) {
  return run_deform(c, s, prec, a, c->stream, P<uint32_t>(c->status));
}

// Everything of a frame up to (and including) the key emission.
// offsets: keep each Gaussian's emission offset (the backward's pair slots), which
// only the key emission produces.
// One scene's share of a frame's Gaussian set: its deformed Gaussians and
// projections sit at [off, off + n) of the work arrays; shift translates the
// scene in the world (composition, Sec. 5.4: G' = {G'_1, ..., G'_n}).
struct FramePart {
  Scene* s;
  long long off;
  float shift[3];
};

long long parts_total(const FramePart* parts, int n_parts) {
  long long n = 0;
  for (int i = 0; i < n_parts; ++i) n += parts[i].s->n;
  return n;
}

// Eq. 5 + Sec. 4.2 + Eq. 6 for one part of a frame into the work arrays at its
// offset, and for a scene with them the colour and opacity heads (App. B) on the
// f_d the deformation leaves.
fs4d_status deform_part(fs4d_ctx* c, Work& w, const FramePart& q, fs4d_precision prec, const float* d_t, float t,
                        cudaStream_t stream, uint32_t* status, void* zero = nullptr, size_t zero_bytes = 0) {
  DeformArgs da = deform_args(q.s, d_t, t, 1, P<float>(w.dmeans) + 3 * q.off, P<float>(w.dquats) + 4 * q.off,
                              P<float>(w.dscales) + 3 * q.off);
  da.zero = static_cast<uint4*>(zero);
  da.zero_n16 = (long long)(zero_bytes / 16);
  // f_d: float32 rows from the FP32 kernel; BF16 tile images from the tensor-core kernel (a part's
  // images may run up to 16 KB past its 256 bytes per Gaussian, into the next part's share, which
  // is written only after this part's heads have read them; the buffer has 16 KB to spare)
  if (q.s->color_heads && prec == FS4D_BF16)
    da.fd_tiles = reinterpret_cast<uint4*>(P<uint8_t>(w.fd) + 256 * (size_t)q.off);
  else if (q.s->color_heads)
    da.fd_out = P<float>(w.fd) + 64 * q.off;
  fs4d_status st = run_deform(c, q.s, prec, da, stream, status);
  if (st != FS4D_OK || !q.s->color_heads) return st;
  ColorArgs ca{};
  ca.n = q.s->n;
  ca.perm = P<uint32_t>(q.s->perm);
  ca.fd = da.fd_out;
  ca.fd_tiles = da.fd_tiles;
  ca.weights = P<float>(q.s->mlp) + q.s->color_off;
  ca.k3 = 3 * q.s->K;
  ca.sh = P<float>(q.s->sh);
  ca.logits = P<float>(q.s->opacity_logits);
  ca.sh_out = P<float>(w.dsh) + 48 * q.off;
  ca.logit_out = P<float>(w.dop) + q.off;
  ca.status = status;
  FS4D_CUDA(c, prec == FS4D_BF16 ? launch_color_heads_bf16(ca, stream) : launch_color_heads(ca, stream));
  return FS4D_OK;
}

// Everything of a frame up to (and including) the key emission, over the union of
// the parts' Gaussians.
// cull: the tile lists may leave out Gaussians that no pixel of the tile blends
// (same image; list positions, and so last-contributor indices, differ).
fs4d_status frame_front(const Env& e, const FramePart* parts, int n_parts, fs4d_precision prec,
                        const fs4d_camera& shape, const fs4d_camera* d_cam, const float* d_t, float t, long long cap,
                        bool report, bool deform, bool offsets, bool cull = false) {
  fs4d_ctx* c = e.c;
  Work& w = *e.w;
  const cudaStream_t stream = e.s;
  const int tx = tiles_of(shape.width), ty = tiles_of(shape.height);
  const int tile_bits = ceil_log2((long long)tx * ty);
  const int N = (int)parts_total(parts, n_parts);
  // every buffer the frame needs at zero, in one allocation (cleared below)
  FrameZero& z = w.z;
  frame_zero_layout(N, tx * ty, cap, sort_passes(tile_bits), static_cast<unsigned char*>(w.zero.p), &z);
  if (z.bytes > w.zero.bytes) return fail(c, FS4D_ERR_INVALID_ARG, "frame work memory was not reserved");
  mark(e, 0);
  for (int i = 0; i < n_parts; ++i)
    if (parts[i].s->color_heads && w.cap_color < N)
      return fail(c, FS4D_ERR_INVALID_ARG, "frame work memory of the colour heads was not reserved");
  // the first deformation kernel clears the frame's zeroed state (no memset of its own)
  const bool fold = deform && n_parts > 0 && parts[0].s->n > 0 && z.bytes % 16 == 0;
  if (!fold) FS4D_CUDA(c, cudaMemsetAsync(w.zero.p, 0, z.bytes, stream));
  if (deform) {
    for (int i = 0; i < n_parts; ++i) {
      fs4d_status st = deform_part(c, w, parts[i], prec, d_t, t, stream, e.status, i == 0 && fold ? w.zero.p : nullptr,
                                   i == 0 && fold ? z.bytes : 0);
      if (st != FS4D_OK) return st;
    }
  }
  mark(e, 1);
  for (int i = 0; i < n_parts; ++i) {
    const FramePart& q = parts[i];
    Scene* s = q.s;
    ProjectArgs pa{};
    pa.n = s->n;
    pa.means = P<float>(w.dmeans) + 3 * q.off; pa.quats = P<float>(w.dquats) + 4 * q.off;
    pa.log_scales = P<float>(w.dscales) + 3 * q.off;
    pa.opacity_logits = P<float>(s->opacity_logits); pa.sh = P<float>(s->sh); pa.sh_degree = s->sh_degree;
    if (s->color_heads) {  // App. B: this frame's deformed colour and opacity
      pa.opacity_logits = P<float>(w.dop) + q.off;
      pa.sh = P<float>(w.dsh) + 48 * q.off;
    }
    pa.cam = cam_params(shape);
    if (e.guard_w > 0) {
      pa.cam.guard_w = e.guard_w;
      pa.cam.guard_h = e.guard_h;
    }
    // world_to_cam applied to X + shift: the translation column absorbs W shift
    for (int r = 0; r < 3; ++r)
      pa.cam.m[4 * r + 3] += pa.cam.m[4 * r] * q.shift[0] + pa.cam.m[4 * r + 1] * q.shift[1] +
                             pa.cam.m[4 * r + 2] * q.shift[2];
    pa.cam_dev = d_cam;
    pa.tiles_x = tx; pa.tiles_y = ty;
    pa.xy = P<float2>(w.xy) + q.off; pa.conic_opacity = P<float4>(w.co) + q.off; pa.rgb = P<float>(w.rgb) + 3 * q.off;
    pa.depth = P<float>(w.depth) + q.off; pa.radius = P<int>(w.radius) + q.off; pa.rect = P<int4>(w.rect) + q.off;
    pa.depth_keys = P<unsigned long long>(w.dkeys) + q.off; pa.depth_vals = P<uint32_t>(w.dvals) + q.off;
    pa.index_base = (uint32_t)q.off;
    pa.depth_hist = z.hist;
    FS4D_CUDA(c, launch_project(pa, stream));
  }
  mark(e, 2);
  // Gaussians in (float32 depth, index) order: the emission order
  bool dalt = false;
  const uint32_t* dsel = nullptr;
  SortWork dsw;
  dsw.hist = z.hist; dsw.lookback = z.dlb; dsw.part_counters = z.counters + 8; dsw.max_parts = z.dparts;
  dsw.prezeroed = true;
  dsw.spin_limit = c->spin_limit;
  dsw.grid_counter = z.counters + 56;  // (words 0..7 emission, 8..24 this sort, 32..48 the pair sort)
  FS4D_CUDA(c, launch_sort(P<unsigned long long>(w.dkeys), P<uint32_t>(w.dvals), P<unsigned long long>(w.dkeys_alt),
                           P<uint32_t>(w.dvals_alt), nullptr, N, 0, 32, true, dsw, e.status, stream, &dalt,
                           &dsel));
  mark(e, 3);
  EmitArgs ea{};
  ea.n = N; ea.order = P<uint32_t>(w.dvals); ea.order_alt = P<uint32_t>(w.dvals_alt); ea.order_sel = dsel;
  ea.depth = P<float>(w.depth); ea.rect = P<int4>(w.rect); ea.tiles_x = tx;
  ea.capacity = cap;
  ea.keys = P<unsigned long long>(w.keys); ea.values = P<uint32_t>(w.values);
  ea.offsets = P<uint32_t>(w.offsets);
  ea.lookback = z.emit_lb;
  ea.part_counter = z.counters;
  ea.num_pairs = z.num_pairs;
  ea.num_pairs_sort = z.num_pairs + 1;
  ea.tile_count = z.tile_count;
  ea.n_tiles = tx * ty;
  ea.status = e.status;
  ea.spin_limit = c->spin_limit;
  ea.report_overflow = report ? 1 : 0;
  w.bmp = use_bitmap(c, w, N, tx * ty, offsets);
  // a frame kept for the backward needs each pair's (key, value) slots; any other
  // sorts one 8-byte (tile | Gaussian index) word per pair (16 instead of 24 bytes
  // per pair per pass)
  w.packed = !w.bmp && !offsets;
  ea.packed = w.packed ? 1 : 0;

  if (e.w == &c->w) c->last_binning = w.bmp ? FS4D_BINNING_BITMAP : FS4D_BINNING_SORT;
  if (w.bmp) {
    // bits per (tile, depth rank) and the projected Gaussians copied into rank order;
    // ranges and launch order from the tile counts; each tile's row read in rank
    // order is its list of depth ranks (no keys: the composite needs none)
    ea.bitmap = P<uint32_t>(w.bitmap);
    ea.words = bitmap_words(N);
    ea.keys = nullptr;
    ea.ranges = P<uint2>(w.ranges);
    ea.tile_order = P<uint32_t>(w.tile_order);
    ea.xy = P<float2>(w.xy); ea.conic_opacity = P<float4>(w.co); ea.rgb = P<float>(w.rgb);
    ea.sorted_xy = P<float2>(w.sxy); ea.sorted_co = P<float4>(w.sco); ea.sorted_rgb = P<float>(w.srgb);
    ea.cull = cull ? 1 : 0;  // bitmap frames only: the emission keeps the full rectangles
    if (w.bmp_dirty) FS4D_CUDA(c, cudaMemsetAsync(w.bitmap.p, 0, w.bitmap.bytes, stream));
    w.bmp_dirty = true;  // until the extraction (which clears every bit it reads) is launched
    FS4D_CUDA(c, launch_mark_tiles(ea, stream));
    FS4D_CUDA(c, launch_tile_scan(z.tile_count, tx * ty, z.num_pairs, P<uint2>(w.ranges), nullptr, 0,
                                  P<uint32_t>(w.tile_order), stream, cap, report ? e.status : nullptr));
    FS4D_CUDA(c, launch_extract_tiles(ea, false, stream));
    w.bmp_dirty = false;
  } else {
    FS4D_CUDA(c, launch_scan_emit(ea, stream));
    // tile ranges and the pair sort's digit histograms straight from the tile counts
    FS4D_CUDA(c, launch_tile_scan(z.tile_count, tx * ty, z.num_pairs, P<uint2>(w.ranges), z.hist,
                                  sort_passes(tile_bits), P<uint32_t>(w.tile_order), stream));
  }
  mark(e, 4);
  return FS4D_OK;
}

fs4d_status frame_front(const Env& e, Scene* s, fs4d_precision prec, const fs4d_camera& shape,
                        const fs4d_camera* d_cam, const float* d_t, float t, long long cap, bool report,
                        bool deform = true, bool offsets = false, bool cull = false) {
  const FramePart part{s, 0, {0.f, 0.f, 0.f}};
  return frame_front(e, &part, 1, prec, shape, d_cam, d_t, t, cap, report, deform, offsets, cull);
}

fs4d_status frame_front(fs4d_ctx* c, Scene* s, fs4d_precision prec, const fs4d_camera& shape,
                        const fs4d_camera* d_cam, const float* d_t, float t, long long cap, bool report,
                        bool offsets = false, bool cull = false) {
  return frame_front(env_of(c), s, prec, shape, d_cam, d_t, t, cap, report, true, offsets, cull);
}

// Sort, ranges and composite with n_dev = the sortable pair count on device.
fs4d_status frame_back(const Env& e, const fs4d_camera& shape, long long n_bound, float* d_image, float* d_t_final,
                       int* d_n_contrib, uint32_t** values_out) {
  fs4d_ctx* c = e.c;
  Work& w = *e.w;
  const int tx = tiles_of(shape.width), ty = tiles_of(shape.height);
  const int tile_bits = ceil_log2((long long)tx * ty);
  const FrameZero& z = w.z;
  const uint32_t* n_dev = z.num_pairs + 1;
  bool alt = false;
  mark(e, 5);
  if (!w.bmp) {
    // pairs arrive in depth order: a stable sort on the tile bits gives (tile, depth, index)
    SortWork psw;
    psw.hist = z.hist; psw.lookback = z.plb; psw.part_counters = z.counters + 32; psw.max_parts = z.pparts;
    psw.prezeroed = true;
    psw.spin_limit = c->spin_limit;
    if (sort_parts(n_bound) > z.pparts) return fail(c, FS4D_ERR_INVALID_ARG, "pair bound above the frame's capacity");
    FS4D_CUDA(c, launch_sort(P<unsigned long long>(w.keys), w.packed ? nullptr : P<uint32_t>(w.values),
                             P<unsigned long long>(w.keys_alt), w.packed ? nullptr : P<uint32_t>(w.values_alt), n_dev,
                             n_bound, 32, tile_bits, true, psw, e.status, e.s, &alt));
  }
  // packed: the Gaussian index is the low word of each sorted 64-bit key
  uint32_t* values = w.packed ? reinterpret_cast<uint32_t*>(alt ? P<unsigned long long>(w.keys_alt)
                                                                : P<unsigned long long>(w.keys))
                              : (alt ? P<uint32_t>(w.values_alt) : P<uint32_t>(w.values));
  if (values_out) *values_out = w.packed ? nullptr : values;
  mark(e, 6);
  // with the bitmap the lists hold depth ranks into the rank-ordered copies
  FS4D_CUDA(c, launch_composite(shape.width, shape.height, P<uint2>(w.ranges), values,
                                w.bmp ? P<float2>(w.sxy) : P<float2>(w.xy), w.bmp ? P<float4>(w.sco) : P<float4>(w.co),
                                w.bmp ? P<float>(w.srgb) : P<float>(w.rgb), d_image, d_t_final, d_n_contrib, e.s,
                                P<uint32_t>(w.tile_order), w.packed ? 2 : 1));
  mark(e, 7);
  return FS4D_OK;
}

fs4d_status frame_back(fs4d_ctx* c, const fs4d_camera& shape, long long n_bound, float* d_image, float* d_t_final,
                       int* d_n_contrib) {
  return frame_back(env_of(c), shape, n_bound, d_image, d_t_final, d_n_contrib, &c->last_values);
}

fs4d_status read_pairs(fs4d_ctx* c, const uint32_t* d_num_pairs, long long* K) {
  FS4D_CUDA(c, cudaMemcpyAsync(c->h_pinned, d_num_pairs, 8, cudaMemcpyDeviceToHost, c->stream));
  FS4D_CUDA(c, cudaStreamSynchronize(c->stream));
  *K = (long long)c->h_pinned[0];
  return FS4D_OK;
}

// One pair-sort pass counts at most 2^30 - 1 pairs (30-bit look-back values).  A
// frame with more pairs renders in horizontal bands of tile rows: each band is a
// frame of its own on the same deformed Gaussians, with the camera's principal
// point moved by the band's offset (a whole number of tiles, so every pixel keeps
// its tile), composited into the band's rows of the image.
constexpr long long kMaxBandPairs = (1ll << 30) - 1;

// Adds the stage times of the pass that just ended (timing on) to c->stage_acc.
fs4d_status add_stage_times(fs4d_ctx* c, bool with_deform) {
  if (!c->timing) return FS4D_OK;
  FS4D_CUDA(c, cudaEventSynchronize(c->ev[7]));
  const int from[6] = {0, 1, 2, 3, 5, 6}, to[6] = {1, 2, 3, 4, 6, 7};
  for (int k = with_deform ? 0 : 1; k < 6; ++k) {
    float ms = 0.f;
    FS4D_CUDA(c, cudaEventElapsedTime(&ms, c->ev[from[k]], c->ev[to[k]]));
    c->stage_acc[k] += ms;
  }
  return FS4D_OK;
}

// Bands of tile rows over the deformed Gaussians already in the work memory.
// n_bands equal bands, or (reuse) the last banded frame's bands of tile rows, so that
// frames of one scene and size are cut alike and render alike.
fs4d_status render_bands(fs4d_ctx* c, Scene* s, fs4d_precision prec, const fs4d_camera* cam, float t, int n_bands,
                         float* d_image, float* d_t_final, int32_t* d_n_contrib, bool reuse = false) {
  const int rows = tiles_of(cam->height), tx = tiles_of(cam->width);
  n_bands = std::max(1, std::min(n_bands, rows));
  std::vector<std::pair<int, int>> todo;  // tile-row ranges [r0, r1), taken from the back
  if (reuse)
    todo.assign(c->band_rows.rbegin(), c->band_rows.rend());
  else
    for (int b = n_bands - 1; b >= 0; --b) todo.push_back({rows * b / n_bands, rows * (b + 1) / n_bands});
  std::vector<std::pair<int, int>> used;
  long long total = 0;
  int done = 0;
  fs4d_status st;
  const bool cull = !d_n_contrib;  // bands are never saved for the backward
  Env be = env_of(c);
  be.guard_w = cam->width;
  be.guard_h = cam->height;
  while (!todo.empty()) {
    const std::pair<int, int> band = todo.back();
    todo.pop_back();
    const int r0 = band.first, r1 = band.second;
    fs4d_camera bc = *cam;
    bc.height = std::min(cam->height, kTile * r1) - kTile * r0;
    bc.cy = cam->cy - (float)(kTile * r0);
    if ((st = ensure_work(c, s->n, tx * (r1 - r0), c->w.cap_pairs)) != FS4D_OK) return st;
    if ((st = frame_front(be, s, prec, bc, nullptr, nullptr, t, c->w.cap_pairs, false, false, false, cull)) != FS4D_OK)
      return st;
    long long K = 0;
    if ((st = read_pairs(c, c->w.z.num_pairs, &K)) != FS4D_OK) return st;
    if (K > c->band_pairs) {
      if (r1 - r0 == 1) return fail(c, FS4D_ERR_CAPACITY, "one tile row of the frame holds more pairs than a band may");
      const int mid = (r0 + r1) / 2;
      todo.push_back({mid, r1});
      todo.push_back({r0, mid});
      continue;
    }
    if (K > c->w.cap_pairs) {
      if ((st = ensure_work(c, s->n, tx * (r1 - r0), std::min(K + K / 4, c->band_pairs))) != FS4D_OK) return st;
      if ((st = frame_front(be, s, prec, bc, nullptr, nullptr, t, c->w.cap_pairs, false, false, false, cull)) !=
          FS4D_OK)
        return st;
    }
    const size_t off = (size_t)kTile * r0 * cam->width;
    if ((st = frame_back(c, bc, K, d_image + 3 * off, d_t_final ? d_t_final + off : nullptr,
                         d_n_contrib ? d_n_contrib + off : nullptr)) != FS4D_OK)
      return st;
    if ((st = add_stage_times(c, false)) != FS4D_OK) return st;
    total += K;
    ++done;
    used.push_back({r0, r1});
  }
  c->last_pairs = total;
  c->last_bands = done;
  // the next frame of this scene and size starts with as many bands, unless one would do
  c->band_scene = s->id; c->band_w = cam->width; c->band_h = cam->height;
  c->band_hint = total > c->band_pairs ? done : 0;
  c->band_rows = used;
  c->stage_acc_valid = c->timing;
  return FS4D_OK;
}

// offsets: the frame will be saved for a backward
fs4d_status render_sync(fs4d_ctx* c, Scene* s, fs4d_precision prec, const fs4d_camera* cam, float t, float* d_image,
                        float* d_t_final, int32_t* d_n_contrib, bool offsets = false) {
  const int n_tiles = tiles_of(cam->width) * tiles_of(cam->height);
  fs4d_status st = ensure_work(c, s->n, n_tiles, c->w.cap_pairs);
  if (st != FS4D_OK) return st;
  if (s->color_heads && (st = ensure_color(c, c->w, c->stream, s->n)) != FS4D_OK) return st;
  std::fill(c->stage_acc, c->stage_acc + 6, 0.f);
  c->stage_acc_valid = false;
  c->last_bands = 1;
  if (!offsets && c->band_hint > 1 && c->band_scene == s->id && c->band_w == cam->width && c->band_h == cam->height) {
    // the last frame of this scene and size needed bands: deform, then bands straight away
    mark(c, 0);
    const FramePart part{s, 0, {0.f, 0.f, 0.f}};
    if ((st = deform_part(c, c->w, part, prec, nullptr, t, c->stream, P<uint32_t>(c->status))) != FS4D_OK) return st;
    mark(c, 1);
    if (c->timing) {
      FS4D_CUDA(c, cudaEventSynchronize(c->ev[1]));
      FS4D_CUDA(c, cudaEventElapsedTime(&c->stage_acc[0], c->ev[0], c->ev[1]));
    }
    return render_bands(c, s, prec, cam, t, c->band_hint, d_image, d_t_final, d_n_contrib, true);
  }
  // lists may drop Gaussians no pixel of their tile blends unless the frame reports
  // list positions (last contributors) or keeps the backward's pair slots
  const bool cull = !offsets && !d_n_contrib;
  st = frame_front(c, s, prec, *cam, nullptr, nullptr, t, c->w.cap_pairs, false, offsets, cull);
  if (st != FS4D_OK) return st;
  long long K = 0;
  if ((st = read_pairs(c, c->w.z.num_pairs, &K)) != FS4D_OK) return st;
  if (K > c->band_pairs) {
    if (offsets) return fail(c, FS4D_ERR_CAPACITY, "a frame saved for the backward must fit one band of tile pairs");
    if ((st = add_stage_times(c, true)) != FS4D_OK) return st;
    // K saturates at 2^32 - 1; a band that still holds too many pairs is split again
    const long long per = std::max(c->band_pairs / 2, 1ll);
    return render_bands(c, s, prec, cam, t, (int)std::min<long long>((K + per - 1) / per, 1 << 20), d_image,
                        d_t_final, d_n_contrib);
  }
  if (K > c->w.cap_pairs) {
    if ((st = ensure_work(c, s->n, n_tiles, std::min(K + K / 4, c->band_pairs))) != FS4D_OK) return st;
    st = frame_front(c, s, prec, *cam, nullptr, nullptr, t, c->w.cap_pairs, false, offsets, cull);
    if (st != FS4D_OK) return st;
  }
  c->last_pairs = K;
  c->last_bands = 1;
  return frame_back(c, *cam, K, d_image, d_t_final, d_n_contrib);
}

// Render with the state the backward needs, into f (its buffers are reused and
// grown when needed, so a frame object can serve one training step after another).
fs4d_status render_into_frame(fs4d_ctx* c, Scene* s, fs4d_precision prec, const fs4d_camera* cam, float t,
                              float* d_image, fs4d_frame* f) {
  const size_t npix = (size_t)cam->width * cam->height;
  if (ensure(f->t_final, 4 * npix) != cudaSuccess || ensure(f->n_contrib, 4 * npix) != cudaSuccess)
    return fail(c, FS4D_ERR_OOM, "render: frame allocation failed");
  fs4d_status st = render_sync(c, s, prec, cam, t, d_image, P<float>(f->t_final), P<int32_t>(f->n_contrib), true);
  if (st != FS4D_OK) return st;
  Work& w = c->w;
  const size_t n = (size_t)s->n, K = (size_t)c->last_pairs;
  const size_t tiles = (size_t)tiles_of(cam->width) * tiles_of(cam->height);
  struct Item {
    DevBuf* dst;
    const void* src;
    size_t bytes;
  } items[] = {{&f->dmeans, w.dmeans.p, 12 * n}, {&f->dquats, w.dquats.p, 16 * n}, {&f->dscales, w.dscales.p, 12 * n},
               {&f->xy, w.xy.p, 8 * n},          {&f->co, w.co.p, 16 * n},         {&f->rgb, w.rgb.p, 12 * n},
               {&f->radius, w.radius.p, 4 * n},  {&f->rect, w.rect.p, 16 * n},     {&f->offsets, w.offsets.p, 4 * n},
               {&f->values, c->last_values, 4 * std::max<size_t>(K, 1)},           {&f->ranges, w.ranges.p, 8 * tiles}};
  for (Item& it : items) {
    if (it.dst->bytes < it.bytes) {
      FS4D_CUDA(c, cudaStreamSynchronize(c->stream));  // the old buffer may still be read
      if (ensure(*it.dst, it.bytes) != cudaSuccess) return fail(c, FS4D_ERR_OOM, "render: frame allocation failed");
    }
    if (cudaMemcpyAsync(it.dst->p, it.src, it.bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
      return fail(c, FS4D_ERR_CUDA, "render: saving the frame failed");
  }
  f->scene = s->id;
  f->cam = *cam;
  f->t = t;
  f->n = s->n;
  f->pairs = c->last_pairs;
  return FS4D_OK;
}

}  // namespace

// ============================================================== C ABI

extern "C" {

fs4d_status fs4d_create(int32_t device, void* cuda_stream, fs4d_ctx** out) {
  if (!out) return FS4D_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FS4D_ERR_INVALID_ARG;
  fs4d_ctx* c = new (std::nothrow) fs4d_ctx();
  if (!c) return FS4D_ERR_OOM;
  c->device = device;
  c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  DeviceGuard g(device);
  if (ensure(c->status, 16) != cudaSuccess || cudaMemset(c->status.p, 0, 16) != cudaSuccess ||
      cudaMallocHost(&c->h_pinned, 16) != cudaSuccess) {
    release(c->status);
    delete c;
    return FS4D_ERR_OOM;
  }
  *out = c;
  return FS4D_OK;
}

fs4d_status fs4d_destroy(fs4d_ctx* c) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (c->server) fs4d_server_destroy(c->server);
  {
    DeviceGuard g(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto& kv : c->scenes) free_scene(kv.second);
    Work& w = c->w;
    DevBuf* all[] = {&w.dmeans, &w.dquats, &w.dscales, &w.xy, &w.co, &w.rgb, &w.depth, &w.radius, &w.rect,
                     &w.offsets, &w.emit_lb, &w.counters, &w.num_pairs, &w.hist, &w.keys, &w.values,
                     &w.keys_alt, &w.values_alt, &w.sort_lb, &w.ranges, &w.tile_count, &w.tile_order, &w.zero, &w.bitmap, &w.sxy, &w.sco, &w.srgb, &w.ts, &w.host_img,
                     &w.grad_pair, &w.gd, &w.acts, &w.wpartial};
    for (DevBuf* b : all) release(*b);
    release(c->status);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    for (int i = 0; i < 8; ++i)
      if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    for (int i = 0; i < 5; ++i)
      if (c->bev[i]) cudaEventDestroy(c->bev[i]);
    if (c->copy_stream) {
      cudaStreamSynchronize(c->copy_stream);
      cudaStreamDestroy(c->copy_stream);
    }
    for (int i = 0; i < 2; ++i) {
      if (c->slot_rendered[i]) cudaEventDestroy(c->slot_rendered[i]);
      if (c->slot_copied[i]) cudaEventDestroy(c->slot_copied[i]);
    }
    if (c->h_pairs) cudaFreeHost(c->h_pairs);
  }
  delete c;
  return FS4D_OK;
}

const char* fs4d_last_error(const fs4d_ctx* c) { return c ? c->err.c_str() : "null context"; }

fs4d_status fs4d_set_stream(fs4d_ctx* c, void* cuda_stream) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  return FS4D_OK;
}

fs4d_status fs4d_set_wait_limit(fs4d_ctx* c, uint32_t polls) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  c->spin_limit = polls == 0 ? kSpinLimit : polls;
  return FS4D_OK;
}

fs4d_status fs4d_check_canaries(fs4d_ctx* c) {
  if (!c) return FS4D_ERR_INVALID_ARG;
#ifdef FS4D_CHECK_BOUNDS
  DeviceGuard g(c->device);
  FS4D_CUDA(c, cudaDeviceSynchronize());
  std::lock_guard<std::mutex> lock(g_canary_mu);
  std::vector<unsigned char> host(kCanaryBytes);
  for (const auto& kv : g_canaries) {
    FS4D_CUDA(c, cudaMemcpy(host.data(), static_cast<unsigned char*>(kv.first) + kv.second, kCanaryBytes,
                            cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < kCanaryBytes; ++i)
      if (host[i] != kCanary)
        return fail(c, FS4D_ERR_CORRUPT, "canary overwritten " + std::to_string(i) + " bytes after a buffer of " +
                                             std::to_string(kv.second) + " bytes");
  }
  return FS4D_OK;
#else
  return fail(c, FS4D_ERR_UNIMPLEMENTED, "check_canaries: built without FS4D_CHECK_BOUNDS");
#endif
}

fs4d_status fs4d_debug_corrupt_canary(fs4d_ctx* c) {
  if (!c) return FS4D_ERR_INVALID_ARG;
#ifdef FS4D_CHECK_BOUNDS
  DeviceGuard g(c->device);
  std::lock_guard<std::mutex> lock(g_canary_mu);
  if (!g_last_buffer) return fail(c, FS4D_ERR_NOT_FOUND, "debug_corrupt_canary: no buffer");
  FS4D_CUDA(c, cudaMemset(static_cast<unsigned char*>(g_last_buffer) + g_canaries[g_last_buffer], 0, 1));
  return FS4D_OK;
#else
  return fail(c, FS4D_ERR_UNIMPLEMENTED, "debug_corrupt_canary: built without FS4D_CHECK_BOUNDS");
#endif
}

fs4d_status fs4d_check_device_status(fs4d_ctx* c) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  FS4D_CUDA(c, cudaMemcpyAsync(c->h_pinned + 2, c->status.p, 4, cudaMemcpyDeviceToHost, c->stream));
  FS4D_CUDA(c, cudaMemsetAsync(c->status.p, 0, 4, c->stream));
  FS4D_CUDA(c, cudaStreamSynchronize(c->stream));
  const uint32_t v = c->h_pinned[2];
  if (v & kStatusTimeout) return fail(c, FS4D_ERR_TIMEOUT, "a bounded device-side wait timed out");
  if (v & kStatusCapacity) return fail(c, FS4D_ERR_CAPACITY, "tile-pair capacity exceeded");
  return FS4D_OK;
}

fs4d_status fs4d_load_scene(fs4d_ctx* c, const fs4d_scene_desc* d, fs4d_scene_id* out) {
  if (!c || !d || !out) return fail(c, FS4D_ERR_INVALID_ARG, "null argument");
  if (d->n < 1 || d->sh_degree < 0 || d->sh_degree > 3 || !d->means || !d->log_scales || !d->quats ||
      !d->opacity_logits || !d->sh || !d->planes || !d->mlp)
    return fail(c, FS4D_ERR_INVALID_ARG, "scene: n >= 1, sh_degree 0..3 and every array are required");
  if (d->n_levels < 1 || d->n_levels > kMaxLevels || d->res_time < 2)
    return fail(c, FS4D_ERR_INVALID_ARG, "scene: 1..4 levels and res_time >= 2 are required");
  for (int l = 0; l < d->n_levels; ++l)
    if (d->res_spatial[l] < 2) return fail(c, FS4D_ERR_INVALID_ARG, "scene: spatial resolution >= 2 required");
  for (int a = 0; a < 3; ++a)
    if (!(d->aabb_max[a] > d->aabb_min[a])) return fail(c, FS4D_ERR_INVALID_ARG, "scene: empty bounding box");
  if (d->mlp_width != kWidth) return fail(c, FS4D_ERR_UNIMPLEMENTED, "scene: only MLP width 64 is supported");
  if (d->color_heads != 0 && d->color_heads != 1)
    return fail(c, FS4D_ERR_INVALID_ARG, "scene: color_heads is 0 or 1");
  if (!deform_fp32_supported(d->feat_dim, d->n_levels))
    return fail(c, FS4D_ERR_UNIMPLEMENTED, "scene: feat_dim must be 16 or 32 with 1..3 levels");
  DeviceGuard g(c->device);
  Scene* s = new Scene();
  s->shape = *d;
  s->shape.means = s->shape.log_scales = s->shape.quats = s->shape.opacity_logits = s->shape.sh = nullptr;
  s->shape.planes = s->shape.mlp = nullptr;
  s->n = d->n;
  s->sh_degree = d->sh_degree;
  s->K = (d->sh_degree + 1) * (d->sh_degree + 1);
  size_t acc = 0;
  const size_t n = (size_t)d->n;
  size_t planes_total;
  plane_geom(*d, s->pg, planes_total);
  s->planes_floats = planes_total;
  const int hin = d->feat_dim * d->n_levels;
  size_t mlp_total;
  src_layers(hin, d->mlp_width, &mlp_total);
  s->color_off = mlp_total;  // the colour and opacity heads follow the eight layers
  s->color_heads = d->color_heads != 0;
  mlp_total = mlp_floats_of(*d);
  s->mlp_floats = mlp_total;
  fs4d_status st;
  auto bail = [&](fs4d_status e) { free_scene(s); return e; };
  if ((st = upload(c, s->means, d->means, 3 * n, &acc)) != FS4D_OK) return bail(st);
  if ((st = upload(c, s->log_scales, d->log_scales, 3 * n, &acc)) != FS4D_OK) return bail(st);
  if ((st = upload(c, s->quats, d->quats, 4 * n, &acc)) != FS4D_OK) return bail(st);
  if ((st = upload(c, s->opacity_logits, d->opacity_logits, n, &acc)) != FS4D_OK) return bail(st);
  if ((st = upload(c, s->sh, d->sh, 3 * n * s->K, &acc)) != FS4D_OK) return bail(st);
  if ((st = upload(c, s->planes, d->planes, planes_total, &acc)) != FS4D_OK) return bail(st);
  std::vector<uint16_t> pb(planes_total);
  for (size_t i = 0; i < planes_total; ++i) pb[i] = f2bf(d->planes[i]);
  if ((st = upload(c, s->planes_bf16, pb.data(), planes_total, &acc)) != FS4D_OK) return bail(st);
  if ((st = upload(c, s->mlp, d->mlp, mlp_total, &acc)) != FS4D_OK) return bail(st);
  std::vector<float> mt = transpose_mlp(d->mlp, hin, d->mlp_width, s->mg);
  if ((st = upload(c, s->mlp_t, mt.data(), mt.size(), &acc)) != FS4D_OK) return bail(st);
  s->bf16_ok = deform_bf16_supported(d->feat_dim, d->n_levels);
  if (s->bf16_ok) {
    std::vector<uint8_t> img;
    std::vector<float> bias;
    build_tc_image(d->mlp, hin, d->mlp_width, s->tg, img, bias);
    if ((st = upload(c, s->tc_ops, img.data(), img.size(), &acc)) != FS4D_OK) return bail(st);
    if ((st = upload(c, s->tc_bias, bias.data(), bias.size(), &acc)) != FS4D_OK) return bail(st);
  }
  {
    std::vector<int4> tab = build_derive_tab(hin, d->mlp_width, s->mg, s->tg, s->bf16_ok);
    if ((st = upload(c, s->derive_tab, tab.data(), tab.size(), &acc)) != FS4D_OK) return bail(st);
  }
  {
    // Work order of the deformation kernels: Gaussians sorted by the 30-bit
    // Morton code of their mean inside the HexPlane box, so that the Gaussians
    // of one warp/CTA gather neighbouring plane cells (outputs keep Gaussian order).
    std::vector<std::pair<uint32_t, uint32_t>> code(n);
    auto spread = [](uint32_t v) {
      v &= 1023u;
      v = (v | (v << 16)) & 0x030000FFu;
      v = (v | (v << 8)) & 0x0300F00Fu;
      v = (v | (v << 4)) & 0x030C30C3u;
      v = (v | (v << 2)) & 0x09249249u;
      return v;
    };
    for (size_t g = 0; g < n; ++g) {
      uint32_t q[3];
      for (int k = 0; k < 3; ++k) {
        const float u = (d->means[3 * g + k] - d->aabb_min[k]) / (d->aabb_max[k] - d->aabb_min[k]);
        q[k] = (uint32_t)std::min(1023.f, std::max(0.f, u * 1023.f));
      }
      code[g] = {spread(q[0]) | (spread(q[1]) << 1) | (spread(q[2]) << 2), (uint32_t)g};
    }
    std::sort(code.begin(), code.end());
    std::vector<uint32_t> perm(n);
    for (size_t i = 0; i < n; ++i) perm[i] = code[i].second;
    if ((st = upload(c, s->perm, perm.data(), n, &acc)) != FS4D_OK) return bail(st);
  }
  s->resident = acc;
  std::lock_guard<std::mutex> lock(c->mu);
  const int id = c->next_id++;
  s->id = id;
  c->scenes[id] = s;
  *out = id;
  return FS4D_OK;
}

fs4d_status fs4d_unload_scene(fs4d_ctx* c, fs4d_scene_id id) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  Scene* s;
  fs4d_status st = get_scene(c, id, &s);
  if (st != FS4D_OK) return st;
  DeviceGuard g(c->device);
  {
    std::lock_guard<std::mutex> lock(c->mu);
    s->dying = true;  // the serving thread launches nothing new on it
  }
  for (int i = 0; i < 200000 && s->refs.load() > 0; ++i) std::this_thread::sleep_for(std::chrono::microseconds(50));
  if (s->refs.load() > 0) {
    std::lock_guard<std::mutex> lock(c->mu);
    s->dying = false;
    return fail(c, FS4D_ERR_TIMEOUT, "unload_scene: serving requests on this scene did not finish");
  }
  cudaStreamSynchronize(c->stream);
  {
    std::lock_guard<std::mutex> lock(c->mu);
    c->scenes.erase(id);
  }
  free_scene(s);
  return FS4D_OK;
}

fs4d_status fs4d_scene_bytes(fs4d_ctx* c, fs4d_scene_id id, int32_t width, int32_t height, float ppg,
                             size_t* resident, size_t* per_frame) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  Scene* s;
  fs4d_status st = get_scene(c, id, &s);
  if (st != FS4D_OK) return st;
  if (resident) *resident = s->resident;
  if (per_frame) {
    const size_t n = (size_t)s->n;
    const size_t pairs = (size_t)(std::max(0.f, ppg) * (float)n) + 4096;
    const size_t tiles = (size_t)tiles_of(width) * tiles_of(height);
    const size_t bmp = bitmap_bytes((int)n, (long long)tiles);
    *per_frame = (bmp <= kBitmapMaxBytes ? bmp + 36 * n : 0) + n * (12 + 16 + 12 + 8 + 16 + 12 + 4 + 4 + 16 + 4 + 24) + pairs * 24 +
                 sort_parts((long long)pairs) * 256 * 4 * kSortMaxPasses + tiles * 8 +
                 (size_t)width * height * 12;
  }
  return FS4D_OK;
}

fs4d_status fs4d_deform(fs4d_ctx* c, fs4d_scene_id id, fs4d_precision prec, const float* h_ts, int32_t n_t,
                        float* d_means, float* d_quats, float* d_log_scales) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (n_t < 1 || !h_ts || !d_means || !d_quats || !d_log_scales)
    return fail(c, FS4D_ERR_INVALID_ARG, "deform: n_t >= 1 and every pointer are required");
  Scene* s;
  fs4d_status st = get_scene(c, id, &s);
  if (st != FS4D_OK) return st;
  DeviceGuard g(c->device);
  if (c->w.ts.bytes < 4 * (size_t)n_t) {
    FS4D_CUDA(c, cudaStreamSynchronize(c->stream));
    FS4D_CUDA(c, ensure(c->w.ts, 4 * (size_t)n_t));
  }
  FS4D_CUDA(c, cudaMemcpyAsync(c->w.ts.p, h_ts, 4 * (size_t)n_t, cudaMemcpyHostToDevice, c->stream));
  DeformArgs a = deform_args(s, P<float>(c->w.ts), 0.f, n_t, d_means, d_quats, d_log_scales);
  return run_deform(c, s, prec, a);
}

namespace {
fs4d_status render_impl(fs4d_ctx* c, fs4d_scene_id id, fs4d_precision prec, const fs4d_camera* cam, float t,
                        float* d_image, float* d_t_final, int32_t* d_n_contrib, fs4d_frame** saved) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (!valid_cam(cam) || !d_image) return fail(c, FS4D_ERR_INVALID_ARG, "render: camera and image are required");
  Scene* s;
  fs4d_status st = get_scene(c, id, &s);
  if (st != FS4D_OK) return st;
  DeviceGuard g(c->device);
  if (!saved) return render_sync(c, s, prec, cam, t, d_image, d_t_final, d_n_contrib);
  *saved = nullptr;
  fs4d_frame* f = new (std::nothrow) fs4d_frame();
  if (!f) return fail(c, FS4D_ERR_OOM, "render: frame allocation failed");
  st = render_into_frame(c, s, prec, cam, t, d_image, f);
  if (st == FS4D_OK && d_t_final)
    st = cudaMemcpyAsync(d_t_final, f->t_final.p, 4 * (size_t)cam->width * cam->height, cudaMemcpyDeviceToDevice,
                         c->stream) == cudaSuccess ? FS4D_OK : fail(c, FS4D_ERR_CUDA, "render: copy of T failed");
  if (st == FS4D_OK && d_n_contrib)
    st = cudaMemcpyAsync(d_n_contrib, f->n_contrib.p, 4 * (size_t)cam->width * cam->height,
                         cudaMemcpyDeviceToDevice, c->stream) == cudaSuccess
             ? FS4D_OK
             : fail(c, FS4D_ERR_CUDA, "render: copy of n_contrib failed");
  if (st != FS4D_OK) {
    fs4d_frame_free(c, f);
    return st;
  }
  *saved = f;
  return FS4D_OK;
}
}  // namespace

fs4d_status fs4d_render(fs4d_ctx* c, fs4d_scene_id id, fs4d_precision prec, const fs4d_camera* cam, float t,
                        float* d_image, float* d_t_final, int32_t* d_n_contrib, fs4d_frame** saved) {
  const unsigned long long before = g_kernel_launches;
  const fs4d_status st = render_impl(c, id, prec, cam, t, d_image, d_t_final, d_n_contrib, saved);
  if (c) c->last_launches = (long long)(g_kernel_launches - before);
  return st;
}

fs4d_status fs4d_render_composed(fs4d_ctx* c, const fs4d_scene_id* ids, const float* h_shifts, int32_t n_scenes,
                                 fs4d_precision prec, const fs4d_camera* cam, float t, float* d_image,
                                 float* d_t_final, int32_t* d_n_contrib) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (!ids || n_scenes < 1 || !valid_cam(cam) || !d_image)
    return fail(c, FS4D_ERR_INVALID_ARG, "render_composed: scenes, camera and image are required");
  std::vector<FramePart> parts;
  long long N = 0;
  for (int i = 0; i < n_scenes; ++i) {
    Scene* s;
    fs4d_status st = get_scene(c, ids[i], &s);
    if (st != FS4D_OK) return st;
    FramePart q{s, N, {0.f, 0.f, 0.f}};
    if (h_shifts)
      for (int k = 0; k < 3; ++k) q.shift[k] = h_shifts[3 * i + k];
    parts.push_back(q);
    N += s->n;
  }
  if (N >= (1ll << 31) - 1) return fail(c, FS4D_ERR_CAPACITY, "render_composed: more than 2^31 - 2 Gaussians");
  DeviceGuard g(c->device);
  const int n_tiles = tiles_of(cam->width) * tiles_of(cam->height);
  fs4d_status st = ensure_work(c, (int)N, n_tiles, c->w.cap_pairs);
  if (st != FS4D_OK) return st;
  for (const FramePart& q : parts)
    if (q.s->color_heads && (st = ensure_color(c, c->w, c->stream, (int)N)) != FS4D_OK) return st;
  c->stage_acc_valid = false;
  st = frame_front(env_of(c), parts.data(), n_scenes, prec, *cam, nullptr, nullptr, t, c->w.cap_pairs, false, true,
                   false, !d_n_contrib);
  if (st != FS4D_OK) return st;
  long long K = 0;
  if ((st = read_pairs(c, c->w.z.num_pairs, &K)) != FS4D_OK) return st;
  if (K > c->band_pairs) return fail(c, FS4D_ERR_CAPACITY, "render_composed: the frame's pairs exceed one band");
  if (K > c->w.cap_pairs) {
    if ((st = ensure_work(c, (int)N, n_tiles, std::min(K + K / 4, c->band_pairs))) != FS4D_OK) return st;
    st = frame_front(env_of(c), parts.data(), n_scenes, prec, *cam, nullptr, nullptr, t, c->w.cap_pairs, false, true,
                     false, !d_n_contrib);
    if (st != FS4D_OK) return st;
  }
  c->last_pairs = K;
  c->last_bands = 1;
  return frame_back(c, *cam, K, d_image, d_t_final, d_n_contrib);
}

fs4d_status fs4d_render_host(fs4d_ctx* c, fs4d_scene_id id, fs4d_precision prec, const fs4d_camera* cam, float t,
                             float* h_image) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (!valid_cam(cam) || !h_image) return fail(c, FS4D_ERR_INVALID_ARG, "render_host: camera and image required");
  Scene* s;
  fs4d_status st = get_scene(c, id, &s);
  if (st != FS4D_OK) return st;
  DeviceGuard g(c->device);
  DevBuf& img = c->w.host_img;
  const size_t bytes = (size_t)cam->width * cam->height * 12;
  if (img.bytes < bytes) {
    FS4D_CUDA(c, cudaStreamSynchronize(c->stream));
    FS4D_CUDA(c, ensure(img, bytes));
  }
  // The whole frame is queued at the current pair capacity and the pair count comes
  // back with the image, so one host synchronisation per frame suffices; a frame
  // whose pairs overflowed the capacity (its image is incomplete) is rendered again
  // with the capacity grown.
  const int n_tiles = tiles_of(cam->width) * tiles_of(cam->height);
  if ((st = ensure_work(c, s->n, n_tiles, c->w.cap_pairs)) != FS4D_OK) return st;
  if (s->color_heads && (st = ensure_color(c, c->w, c->stream, s->n)) != FS4D_OK) return st;
  const long long cap = c->w.cap_pairs;
  if ((st = frame_front(c, s, prec, *cam, nullptr, nullptr, t, cap, false, false, true)) != FS4D_OK) return st;
  if ((st = frame_back(c, *cam, cap, P<float>(img), nullptr, nullptr)) != FS4D_OK) return st;
  FS4D_CUDA(c, cudaMemcpyAsync(c->h_pinned, c->w.z.num_pairs, 8, cudaMemcpyDeviceToHost, c->stream));
  FS4D_CUDA(c, cudaMemcpyAsync(h_image, img.p, bytes, cudaMemcpyDeviceToHost, c->stream));
  FS4D_CUDA(c, cudaStreamSynchronize(c->stream));
  const long long K = (long long)c->h_pinned[0];
  c->last_pairs = K;
  c->last_bands = 1;
  if (K <= cap) return FS4D_OK;
  st = render_sync(c, s, prec, cam, t, P<float>(img), nullptr, nullptr);
  if (st != FS4D_OK) return st;
  FS4D_CUDA(c, cudaMemcpyAsync(h_image, img.p, bytes, cudaMemcpyDeviceToHost, c->stream));
  FS4D_CUDA(c, cudaStreamSynchronize(c->stream));
  return FS4D_OK;
}

fs4d_status fs4d_render_host_batch(fs4d_ctx* c, fs4d_scene_id id, fs4d_precision prec, const fs4d_camera* cams,
                                   const float* ts, int32_t n, float* const* h_images) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (n < 1 || !cams || !ts || !h_images) return fail(c, FS4D_ERR_INVALID_ARG, "render_host_batch: bad argument");
  for (int k = 0; k < n; ++k)
    if (!valid_cam(&cams[k]) || !h_images[k] || cams[k].width != cams[0].width || cams[k].height != cams[0].height)
      return fail(c, FS4D_ERR_INVALID_ARG, "render_host_batch: frames need valid cameras of one size and images");
  Scene* s;
  fs4d_status st = get_scene(c, id, &s);
  if (st != FS4D_OK) return st;
  DeviceGuard g(c->device);
  const size_t bytes = (size_t)cams[0].width * cams[0].height * 12;
  DevBuf& img = c->w.host_img;  // two slots: a frame renders into one while the other is copied out
  if (img.bytes < 2 * bytes || c->h_pairs_cap < n || !c->copy_stream) {
    FS4D_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->copy_stream) FS4D_CUDA(c, cudaStreamSynchronize(c->copy_stream));
    FS4D_CUDA(c, ensure(img, 2 * bytes));
    if (c->h_pairs_cap < n) {
      if (c->h_pairs) cudaFreeHost(c->h_pairs);
      c->h_pairs = nullptr;
      c->h_pairs_cap = 0;
      FS4D_CUDA(c, cudaMallocHost(&c->h_pairs, sizeof(unsigned long long) * (size_t)n));
      c->h_pairs_cap = n;
    }
    if (!c->copy_stream) {
      FS4D_CUDA(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
      for (int i = 0; i < 2; ++i) {
        FS4D_CUDA(c, cudaEventCreateWithFlags(&c->slot_rendered[i], cudaEventDisableTiming));
        FS4D_CUDA(c, cudaEventCreateWithFlags(&c->slot_copied[i], cudaEventDisableTiming));
      }
    }
  }
  const int n_tiles = tiles_of(cams[0].width) * tiles_of(cams[0].height);
  if ((st = ensure_work(c, s->n, n_tiles, c->w.cap_pairs)) != FS4D_OK) return st;
  if (s->color_heads && (st = ensure_color(c, c->w, c->stream, s->n)) != FS4D_OK) return st;
  const long long cap = c->w.cap_pairs;
  float* slot_img[2] = {P<float>(img), P<float>(img) + bytes / 4};
  for (int k = 0; k < n; ++k) {
    const int sl = k & 1;
    // the slot's previous image (frame k - 2) must be on the host before it is overwritten
    if (k >= 2) FS4D_CUDA(c, cudaStreamWaitEvent(c->stream, c->slot_copied[sl], 0));
    if ((st = frame_front(c, s, prec, cams[k], nullptr, nullptr, ts[k], cap, false, false, true)) != FS4D_OK)
      return st;
    if ((st = frame_back(c, cams[k], cap, slot_img[sl], nullptr, nullptr)) != FS4D_OK) return st;
    // (the count lives in the frame's zeroed state: read before the next frame clears it)
    FS4D_CUDA(c, cudaMemcpyAsync(&c->h_pairs[k], c->w.z.num_pairs, 8, cudaMemcpyDeviceToHost, c->stream));
    FS4D_CUDA(c, cudaEventRecord(c->slot_rendered[sl], c->stream));
    FS4D_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->slot_rendered[sl], 0));
    FS4D_CUDA(c, cudaMemcpyAsync(h_images[k], slot_img[sl], bytes, cudaMemcpyDeviceToHost, c->copy_stream));
    FS4D_CUDA(c, cudaEventRecord(c->slot_copied[sl], c->copy_stream));
  }
  FS4D_CUDA(c, cudaStreamSynchronize(c->stream));
  FS4D_CUDA(c, cudaStreamSynchronize(c->copy_stream));
  // frames whose pairs overflowed the capacity are rendered again (capacity grown)
  for (int k = 0; k < n; ++k) {
    const long long K = (long long)(c->h_pairs[k] & 0xffffffffull);
    c->last_pairs = K;
    c->last_bands = 1;
    if (K <= cap) continue;
    if ((st = render_sync(c, s, prec, &cams[k], ts[k], P<float>(img), nullptr, nullptr)) != FS4D_OK) return st;
    FS4D_CUDA(c, cudaMemcpyAsync(h_images[k], img.p, bytes, cudaMemcpyDeviceToHost, c->stream));
    FS4D_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return FS4D_OK;
}

fs4d_status fs4d_reserve(fs4d_ctx* c, fs4d_scene_id id, int32_t width, int32_t height, int64_t pair_capacity) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (width <= 0 || height <= 0 || pair_capacity < 0) return fail(c, FS4D_ERR_INVALID_ARG, "reserve: bad size");
  Scene* s;
  fs4d_status st = get_scene(c, id, &s);
  if (st != FS4D_OK) return st;
  DeviceGuard g(c->device);
  st = ensure_work(c, s->n, tiles_of(width) * tiles_of(height), pair_capacity);
  if (st == FS4D_OK && s->color_heads) st = ensure_color(c, c->w, c->stream, s->n);
  if (st != FS4D_OK) return st;
  s->reserved_pairs = pair_capacity;
  s->reserved_w = width;
  s->reserved_h = height;
  return FS4D_OK;
}

namespace {
fs4d_status render_async_impl(fs4d_ctx* c, fs4d_scene_id id, fs4d_precision prec, const fs4d_camera* shape,
                              const fs4d_camera* d_cam, const float* d_t, float* d_image) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (!valid_cam(shape) || !d_cam || !d_t || !d_image)
    return fail(c, FS4D_ERR_INVALID_ARG, "render_async: shape, device camera, device t and image are required");
  Scene* s;
  fs4d_status st = get_scene(c, id, &s);
  if (st != FS4D_OK) return st;
  const int n_tiles = tiles_of(shape->width) * tiles_of(shape->height);
  if (s->reserved_pairs <= 0 || c->w.cap_pairs < s->reserved_pairs || c->w.cap_tiles < n_tiles || c->w.cap_n < s->n)
    return fail(c, FS4D_ERR_INVALID_ARG, "render_async: call fs4d_reserve for this scene and size first");
  DeviceGuard g(c->device);
  const long long cap = s->reserved_pairs;
  c->stage_acc_valid = false;  // (a banded frame's sums no longer describe the last frame)
  st = frame_front(c, s, prec, *shape, d_cam, d_t, 0.f, cap, true, false, true);
  if (st != FS4D_OK) return st;
  return frame_back(c, *shape, cap, d_image, nullptr, nullptr);
}
}  // namespace

fs4d_status fs4d_render_async(fs4d_ctx* c, fs4d_scene_id id, fs4d_precision prec, const fs4d_camera* shape,
                              const fs4d_camera* d_cam, const float* d_t, float* d_image) {
  const unsigned long long before = g_kernel_launches;
  const fs4d_status st = render_async_impl(c, id, prec, shape, d_cam, d_t, d_image);
  if (c) c->last_launches = (long long)(g_kernel_launches - before);
  return st;
}

fs4d_status fs4d_set_stage_timing(fs4d_ctx* c, int32_t enable) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  if (enable && !c->ev[0]) {
    for (int i = 0; i < 8; ++i) FS4D_CUDA(c, cudaEventCreate(&c->ev[i]));
    for (int i = 0; i < 5; ++i) FS4D_CUDA(c, cudaEventCreate(&c->bev[i]));
  }
  c->timing = enable != 0;
  return FS4D_OK;
}

fs4d_status fs4d_stage_times(fs4d_ctx* c, float* h_ms) {
  if (!c || !h_ms) return FS4D_ERR_INVALID_ARG;
  if (!c->ev[0]) return fail(c, FS4D_ERR_INVALID_ARG, "stage_times: timing was never enabled");
  DeviceGuard g(c->device);
  if (c->stage_acc_valid) {  // a frame rendered in bands: the sum over its passes
    for (int k = 0; k < 6; ++k) h_ms[k] = c->stage_acc[k];
    return FS4D_OK;
  }
  FS4D_CUDA(c, cudaEventSynchronize(c->ev[7]));
  const int from[6] = {0, 1, 2, 3, 5, 6}, to[6] = {1, 2, 3, 4, 6, 7};
  for (int k = 0; k < 6; ++k) FS4D_CUDA(c, cudaEventElapsedTime(&h_ms[k], c->ev[from[k]], c->ev[to[k]]));
  return FS4D_OK;
}

fs4d_status fs4d_backward_times(fs4d_ctx* c, float* h_ms) {
  if (!c || !h_ms) return FS4D_ERR_INVALID_ARG;
  if (!c->bev[0]) return fail(c, FS4D_ERR_INVALID_ARG, "backward_times: timing was never enabled");
  DeviceGuard g(c->device);
  FS4D_CUDA(c, cudaEventSynchronize(c->bev[4]));
  for (int k = 0; k < 4; ++k) FS4D_CUDA(c, cudaEventElapsedTime(&h_ms[k], c->bev[k], c->bev[k + 1]));
  return FS4D_OK;
}

static fs4d_status backward_impl(fs4d_ctx* c, fs4d_frame* f, const float* d_dl_dimage, const fs4d_grads* gr,
                                 const fs4d_view_stats* stats) {
  NvtxScope nvtx_scope("fs4d:backward");
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (!f || !d_dl_dimage || !gr) return fail(c, FS4D_ERR_INVALID_ARG, "render_backward: frame, dL/dI, grads needed");
  if (stats && (!stats->grad_norm_sum || !stats->visible))
    return fail(c, FS4D_ERR_INVALID_ARG, "render_backward: both statistics arrays are needed");
  Scene* s;
  fs4d_status st = get_scene(c, f->scene, &s);
  if (st != FS4D_OK) return st;
  if (s->color_heads)
    return fail(c, FS4D_ERR_UNIMPLEMENTED, "render_backward: no backward through the colour and opacity heads");
  if (s->n != f->n) return fail(c, FS4D_ERR_INVALID_ARG, "render_backward: the scene changed size since the frame");
  DeviceGuard g(c->device);
  Work& w = c->w;
  const long long n = s->n, K = f->pairs;
  const int hin = s->mg.hin;
  const size_t act_floats = (size_t)n * (hin + 64 + 64 + 192 + 10 + 192 + 64 + 64);
  size_t wtot = 0;
  {
    size_t tot_floats;
    auto Ls = src_layers(hin, kWidth, &tot_floats);
    wtot = (size_t)tot_floats;  // every layer's O*I + O entries
  }
  const size_t wp = (size_t)wgrad_chunks(n) * wtot;
  if (w.grad_pair.bytes < 4 * kPairStride * (size_t)std::max(K, 1ll) || w.gd.bytes < 40 * (size_t)n ||
      w.acts.bytes < 4 * act_floats || w.wpartial.bytes < 4 * wp) {
    FS4D_CUDA(c, cudaStreamSynchronize(c->stream));
    FS4D_CUDA(c, ensure(w.grad_pair, 4 * kPairStride * (size_t)std::max(K, 1ll)));
    FS4D_CUDA(c, ensure(w.gd, 40 * (size_t)n));
    FS4D_CUDA(c, ensure(w.acts, 4 * act_floats));
    FS4D_CUDA(c, ensure(w.wpartial, 4 * wp));
  }
  const int tx = tiles_of(f->cam.width);
  auto bmark = [&](int i) {
    if (c->timing) cudaEventRecord(c->bev[i], c->stream);
  };
  bmark(0);
  // 1. compositing backward into per-pair slots
  FS4D_CUDA(c, cudaMemsetAsync(w.grad_pair.p, 0, 4 * kPairStride * (size_t)std::max(K, 1ll), c->stream));
  CompositeBwdArgs cb{};
  cb.width = f->cam.width; cb.height = f->cam.height; cb.tiles_x = tx;
  cb.ranges = P<uint2>(f->ranges); cb.values = P<uint32_t>(f->values);
  cb.xy = P<float2>(f->xy); cb.conic_opacity = P<float4>(f->co); cb.rgb = P<float>(f->rgb);
  cb.rect = P<int4>(f->rect); cb.offsets = P<uint32_t>(f->offsets);
  cb.t_final = P<float>(f->t_final); cb.n_contrib = P<int>(f->n_contrib);
  cb.dl_dimage = d_dl_dimage; cb.grad_pair = P<float>(w.grad_pair);
  FS4D_CUDA(c, launch_composite_bwd(cb, c->stream));
  bmark(1);
  // 2. projection, SH and Eq. 6 identity part
  ProjectBwdArgs pb{};
  pb.n = (int)n;
  pb.means = P<float>(f->dmeans); pb.quats = P<float>(f->dquats); pb.log_scales = P<float>(f->dscales);
  pb.sh = P<float>(s->sh); pb.sh_degree = s->sh_degree; pb.cam = cam_params(f->cam);
  pb.conic_opacity = P<float4>(f->co); pb.radius = P<int>(f->radius); pb.rect = P<int4>(f->rect);
  pb.offsets = P<uint32_t>(f->offsets); pb.grad_pair = P<float>(w.grad_pair); pb.gd = P<float>(w.gd);
  pb.g_means = gr->means; pb.g_quats = gr->quats; pb.g_log_scales = gr->log_scales;
  pb.g_opacity = gr->opacity_logits; pb.g_sh = gr->sh;
  if (stats) {
    pb.stat_grad = stats->grad_norm_sum;
    pb.stat_visible = stats->visible;
  }
  FS4D_CUDA(c, launch_project_bwd(pb, c->stream));
  bmark(2);
  // 3. MLP heads, phi_d and HexPlane sampling (float32 recompute of the deformation)
  MlpBwdArgs mb{};
  mb.f = deform_args(s, nullptr, f->t, 1, nullptr, nullptr, nullptr);
  mb.gd = P<float>(w.gd);
  float* A = P<float>(w.acts);
  mb.act.fh = A; A += (size_t)n * hin;
  mb.act.a1 = A; A += (size_t)n * 64;
  mb.act.fd = A; A += (size_t)n * 64;
  mb.act.hid = A; A += (size_t)n * 192;
  mb.act.dout = A; A += (size_t)n * 10;
  mb.act.dh = A; A += (size_t)n * 192;
  mb.act.d2 = A; A += (size_t)n * 64;
  mb.act.d1 = A;
  mb.g_planes = gr->planes;
  mb.g_means = gr->means;
  FS4D_CUDA(c, launch_mlp_bwd(mb, c->stream));
  bmark(3);
  // 4. weight gradients, deterministic two-stage reductions, source layout
  if (gr->mlp) {
    size_t tot;
    auto L = src_layers(hin, kWidth, &tot);
    const int col0[3] = {0, 3, 7};
    WgradArgs wa{};
    wa.n = n;
    wa.partial = P<float>(w.wpartial);
    auto add = [&](const float* D, const float* X, int O, int I, const SrcLayer& l) {
      wa.l[wa.n_layers++] = WgradLayer{D, X, O, I, gr->mlp + l.w, gr->mlp + l.b, 0};
    };
    add(mb.act.d1, mb.act.fh, 64, hin, L[0]);
    add(mb.act.d2, mb.act.a1, 64, 64, L[1]);
    for (int h = 0; h < 3; ++h) {
      add(mb.act.dh + (size_t)64 * h * n, mb.act.fd, 64, 64, L[2 + 2 * h]);
      add(mb.act.dout + (size_t)col0[h] * n, mb.act.hid + (size_t)64 * h * n, L[3 + 2 * h].out, 64, L[3 + 2 * h]);
    }
    FS4D_CUDA(c, launch_wgrad(wa, c->stream));
  }
  bmark(4);
  return FS4D_OK;
}

fs4d_status fs4d_render_backward(fs4d_ctx* c, fs4d_frame* f, const float* d_dl_dimage, const fs4d_grads* gr) {
  return backward_impl(c, f, d_dl_dimage, gr, nullptr);
}

fs4d_status fs4d_render_backward_stats(fs4d_ctx* c, fs4d_frame* f, const float* d_dl_dimage, const fs4d_grads* gr,
                                       const fs4d_view_stats* stats) {
  if (c && !stats) return fail(c, FS4D_ERR_INVALID_ARG, "render_backward_stats: statistics needed");
  return backward_impl(c, f, d_dl_dimage, gr, stats);
}

fs4d_status fs4d_frame_free(fs4d_ctx* c, fs4d_frame* f) {
  if (!f) return FS4D_OK;
  {
    DeviceGuard g(c ? c->device : 0);
    if (c) cudaStreamSynchronize(c->stream);
    DevBuf* all[] = {&f->dmeans, &f->dquats, &f->dscales, &f->xy, &f->co, &f->rgb, &f->radius,
                     &f->rect, &f->offsets, &f->values, &f->ranges, &f->t_final, &f->n_contrib};
    for (DevBuf* b : all) release(*b);
  }
  delete f;
  return FS4D_OK;
}

fs4d_status fs4d_update_scene(fs4d_ctx* c, fs4d_scene_id id, const fs4d_scene_desc* d, int32_t on_device) {
  if (!c || !d) return FS4D_ERR_INVALID_ARG;
  Scene* s;
  fs4d_status st = get_scene(c, id, &s);
  if (st != FS4D_OK) return st;
  if (d->n != s->n || d->sh_degree != s->sh_degree || d->n_levels != s->pg.n_levels || d->feat_dim != s->pg.feat_dim ||
      d->res_time != s->pg.res_time || d->mlp_width != kWidth || (d->color_heads != 0) != s->color_heads)
    return fail(c, FS4D_ERR_INVALID_ARG, "update_scene: shapes must match the loaded scene");
  DeviceGuard g(c->device);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const size_t n = (size_t)s->n;
  struct Item {
    DevBuf* dst;
    const float* src;
    size_t floats;
  } items[] = {{&s->means, d->means, 3 * n},         {&s->log_scales, d->log_scales, 3 * n},
               {&s->quats, d->quats, 4 * n},         {&s->opacity_logits, d->opacity_logits, n},
               {&s->sh, d->sh, 3 * n * s->K},        {&s->planes, d->planes, s->planes_floats},
               {&s->mlp, d->mlp, s->mlp_floats}};
  for (Item& it : items) {
    if (!it.src) continue;
    FS4D_CUDA(c, cudaMemcpyAsync(it.dst->p, it.src, 4 * it.floats, kind, c->stream));
  }
  // derived copies: BF16 planes and the two MLP layouts (small; prepared on the host)
  FS4D_CUDA(c, cudaStreamSynchronize(c->stream));
  std::vector<float> planes(s->planes_floats), mlp(s->mlp_floats);
  FS4D_CUDA(c, cudaMemcpy(planes.data(), s->planes.p, 4 * planes.size(), cudaMemcpyDeviceToHost));
  FS4D_CUDA(c, cudaMemcpy(mlp.data(), s->mlp.p, 4 * mlp.size(), cudaMemcpyDeviceToHost));
  std::vector<uint16_t> pb(planes.size());
  for (size_t i = 0; i < planes.size(); ++i) pb[i] = f2bf(planes[i]);
  FS4D_CUDA(c, cudaMemcpy(s->planes_bf16.p, pb.data(), 2 * pb.size(), cudaMemcpyHostToDevice));
  std::vector<float> mt = transpose_mlp(mlp.data(), s->mg.hin, kWidth, s->mg);
  FS4D_CUDA(c, cudaMemcpy(s->mlp_t.p, mt.data(), 4 * mt.size(), cudaMemcpyHostToDevice));
  if (s->bf16_ok) {
    std::vector<uint8_t> img;
    std::vector<float> bias;
    build_tc_image(mlp.data(), s->mg.hin, kWidth, s->tg, img, bias);
    FS4D_CUDA(c, cudaMemcpy(s->tc_ops.p, img.data(), img.size(), cudaMemcpyHostToDevice));
    FS4D_CUDA(c, cudaMemcpy(s->tc_bias.p, bias.data(), 4 * bias.size(), cudaMemcpyHostToDevice));
  }
  return FS4D_OK;
}

fs4d_status fs4d_frame_pairs(const fs4d_frame* f, int64_t* pairs) {
  if (!f || !pairs) return FS4D_ERR_INVALID_ARG;
  *pairs = f->pairs;
  return FS4D_OK;
}

fs4d_status fs4d_set_binning(fs4d_ctx* c, int32_t mode) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (mode != FS4D_BINNING_AUTO && mode != FS4D_BINNING_SORT)
    return fail(c, FS4D_ERR_INVALID_ARG, "set_binning: mode must be FS4D_BINNING_AUTO or FS4D_BINNING_SORT");
  c->binning = mode;
  return FS4D_OK;
}

fs4d_status fs4d_last_binning(const fs4d_ctx* c, int32_t* mode) {
  if (!c || !mode) return FS4D_ERR_INVALID_ARG;
  *mode = c->last_binning;
  return FS4D_OK;
}

fs4d_status fs4d_set_band_pairs(fs4d_ctx* c, int64_t max_pairs) {
  if (!c || max_pairs < 0) return FS4D_ERR_INVALID_ARG;
  c->band_pairs = max_pairs == 0 ? kMaxBandPairs : std::min<long long>(max_pairs, kMaxBandPairs);
  c->band_hint = 0;
  return FS4D_OK;
}

fs4d_status fs4d_last_bands(const fs4d_ctx* c, int32_t* bands) {
  if (!c || !bands) return FS4D_ERR_INVALID_ARG;
  *bands = c->last_bands;
  return FS4D_OK;
}

fs4d_status fs4d_last_launches(const fs4d_ctx* c, int64_t* launches) {
  if (!c || !launches) return FS4D_ERR_INVALID_ARG;
  *launches = c->last_launches;
  return FS4D_OK;
}

fs4d_status fs4d_last_pairs(const fs4d_ctx* c, int64_t* pairs) {
  if (!c || !pairs) return FS4D_ERR_INVALID_ARG;
  *pairs = c->last_pairs;
  return FS4D_OK;
}

// ------------------------------------------------------------------ stages

fs4d_status fs4d_project(fs4d_ctx* c, int32_t n, const float* d_means, const float* d_quats,
                         const float* d_log_scales, const float* d_opacity_logits, const float* d_sh,
                         int32_t sh_degree, const fs4d_camera* cam, const fs4d_projected* out) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (n < 0 || !valid_cam(cam) || !out || sh_degree < 0 || sh_degree > 3 ||
      (n > 0 && (!d_means || !d_quats || !d_log_scales || !d_opacity_logits || !d_sh || !out->xy ||
                 !out->conic_opacity || !out->rgb || !out->depth || !out->radius || !out->rect)))
    return fail(c, FS4D_ERR_INVALID_ARG, "project: bad argument");
  DeviceGuard g(c->device);
  ProjectArgs pa{};
  pa.n = n; pa.means = d_means; pa.quats = d_quats; pa.log_scales = d_log_scales;
  pa.opacity_logits = d_opacity_logits; pa.sh = d_sh; pa.sh_degree = sh_degree;
  pa.cam = cam_params(*cam); pa.cam_dev = nullptr;
  pa.tiles_x = tiles_of(cam->width); pa.tiles_y = tiles_of(cam->height);
  pa.xy = reinterpret_cast<float2*>(out->xy); pa.conic_opacity = reinterpret_cast<float4*>(out->conic_opacity);
  pa.rgb = out->rgb; pa.depth = out->depth; pa.radius = out->radius; pa.rect = reinterpret_cast<int4*>(out->rect);
  FS4D_CUDA(c, launch_project(pa, c->stream));
  return FS4D_OK;
}

fs4d_status fs4d_bin_sort(fs4d_ctx* c, int32_t n, const float* d_depth, const int32_t* d_rect, int32_t tiles_x,
                          int32_t tiles_y, int64_t capacity, uint64_t* d_keys, uint32_t* d_values,
                          uint32_t* d_ranges, int64_t* h_num_pairs) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (n < 0 || tiles_x < 1 || tiles_y < 1 || (long long)tiles_x * tiles_y > (1ll << 31) || capacity < 0 ||
      !h_num_pairs || !d_ranges || (n > 0 && (!d_depth || !d_rect)) || (capacity > 0 && (!d_keys || !d_values)))
    return fail(c, FS4D_ERR_INVALID_ARG, "bin_sort: bad argument");
  DeviceGuard g(c->device);
  const int n_tiles = tiles_x * tiles_y;
  fs4d_status st = ensure_work(c, std::max(n, 1), n_tiles, capacity);
  if (st != FS4D_OK) return st;
  Work& w = c->w;
  const int tile_bits = ceil_log2(n_tiles);
  // emission order: Gaussians sorted by (float32 depth, index)
  FS4D_CUDA(c, launch_depth_keys(d_depth, n, P<unsigned long long>(w.dkeys), P<uint32_t>(w.dvals), c->stream));
  bool dalt = false;
  const uint32_t* dsel = nullptr;
  FS4D_CUDA(c, launch_sort(P<unsigned long long>(w.dkeys), P<uint32_t>(w.dvals), P<unsigned long long>(w.dkeys_alt),
                           P<uint32_t>(w.dvals_alt), nullptr, n, 0, 32, false, sort_work(c), P<uint32_t>(c->status),
                           c->stream, &dalt, &dsel));
  FS4D_CUDA(c, cudaMemsetAsync(w.counters.p, 0, 4 * kEmitCounters, c->stream));
  FS4D_CUDA(c, cudaMemsetAsync(w.num_pairs.p, 0, 16, c->stream));
  FS4D_CUDA(c, cudaMemsetAsync(w.tile_count.p, 0, 4 * (size_t)n_tiles, c->stream));
  FS4D_CUDA(c, cudaMemsetAsync(w.emit_lb.p, 0, 8 * (size_t)emit_parts(std::max(n, 1)), c->stream));
  EmitArgs ea{};
  ea.n = n; ea.order = P<uint32_t>(w.dvals); ea.order_alt = P<uint32_t>(w.dvals_alt); ea.order_sel = dsel;
  ea.depth = d_depth; ea.rect = reinterpret_cast<const int4*>(d_rect); ea.tiles_x = tiles_x;
  ea.capacity = capacity;
  ea.keys = reinterpret_cast<unsigned long long*>(d_keys); ea.values = d_values;
  ea.offsets = P<uint32_t>(w.offsets);
  ea.lookback = P<unsigned long long>(w.emit_lb);
  ea.part_counter = P<uint32_t>(w.counters);
  ea.num_pairs = P<uint32_t>(w.num_pairs);
  ea.num_pairs_sort = P<uint32_t>(w.num_pairs) + 1;
  ea.tile_count = P<uint32_t>(w.tile_count);
  ea.n_tiles = n_tiles;
  ea.status = P<uint32_t>(c->status);
  ea.spin_limit = c->spin_limit;
  ea.report_overflow = 0;
  const bool bmp = use_bitmap(c, w, n, n_tiles, false);
  c->last_binning = bmp ? FS4D_BINNING_BITMAP : FS4D_BINNING_SORT;
  if (bmp) {
    ea.bitmap = P<uint32_t>(w.bitmap);
    ea.words = bitmap_words(n);
    ea.ranges = reinterpret_cast<const uint2*>(d_ranges);
    if (w.bmp_dirty) FS4D_CUDA(c, cudaMemsetAsync(w.bitmap.p, 0, w.bitmap.bytes, c->stream));
    w.bmp_dirty = true;
    FS4D_CUDA(c, launch_mark_tiles(ea, c->stream));
    FS4D_CUDA(c, launch_tile_scan(P<uint32_t>(w.tile_count), n_tiles, P<uint32_t>(w.num_pairs),
                                  reinterpret_cast<uint2*>(d_ranges), nullptr, 0, nullptr, c->stream, capacity));
    FS4D_CUDA(c, launch_extract_tiles(ea, true, c->stream));  // also clears the bitmap when the pairs overflow
    w.bmp_dirty = false;
  } else {
    FS4D_CUDA(c, launch_scan_emit(ea, c->stream));
    FS4D_CUDA(c, launch_tile_scan(P<uint32_t>(w.tile_count), n_tiles, P<uint32_t>(w.num_pairs),
                                  reinterpret_cast<uint2*>(d_ranges), P<uint32_t>(w.hist), sort_passes(tile_bits),
                                  nullptr, c->stream));
  }
  long long K = 0;
  if ((st = read_pairs(c, P<uint32_t>(w.num_pairs), &K)) != FS4D_OK) return st;
  *h_num_pairs = K;
  if (K > capacity) {
    return fail(c, FS4D_ERR_CAPACITY, "bin_sort: " + std::to_string(K) + " pairs exceed the capacity");
  }
  if (bmp) return FS4D_OK;
  bool alt = false;
  FS4D_CUDA(c, launch_sort(reinterpret_cast<unsigned long long*>(d_keys), d_values, P<unsigned long long>(w.keys_alt),
                           P<uint32_t>(w.values_alt), nullptr, K, 32, tile_bits, true, sort_work(c),
                           P<uint32_t>(c->status), c->stream, &alt));
  if (alt && K > 0) {
    FS4D_CUDA(c, cudaMemcpyAsync(d_keys, w.keys_alt.p, 8 * (size_t)K, cudaMemcpyDeviceToDevice, c->stream));
    FS4D_CUDA(c, cudaMemcpyAsync(d_values, w.values_alt.p, 4 * (size_t)K, cudaMemcpyDeviceToDevice, c->stream));
  }
  return FS4D_OK;
}

fs4d_status fs4d_sort_pairs(fs4d_ctx* c, int64_t n, int32_t key_bits, uint64_t* d_keys, uint32_t* d_values) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (n < 0 || key_bits < 1 || key_bits > 64 || (n > 0 && (!d_keys || !d_values)) || n >= (1ll << 30))
    return fail(c, FS4D_ERR_INVALID_ARG, "sort_pairs: bad argument");
  if (n == 0) return FS4D_OK;
  DeviceGuard g(c->device);
  fs4d_status st = ensure_work(c, 1, 1, n);
  if (st != FS4D_OK) return st;
  Work& w = c->w;
  bool alt = false;
  FS4D_CUDA(c, launch_sort(reinterpret_cast<unsigned long long*>(d_keys), d_values, P<unsigned long long>(w.keys_alt),
                           P<uint32_t>(w.values_alt), nullptr, n, 0, key_bits, false, sort_work(c),
                           P<uint32_t>(c->status), c->stream, &alt));
  if (alt) {
    FS4D_CUDA(c, cudaMemcpyAsync(d_keys, w.keys_alt.p, 8 * (size_t)n, cudaMemcpyDeviceToDevice, c->stream));
    FS4D_CUDA(c, cudaMemcpyAsync(d_values, w.values_alt.p, 4 * (size_t)n, cudaMemcpyDeviceToDevice, c->stream));
  }
  return FS4D_OK;
}

fs4d_status fs4d_composite(fs4d_ctx* c, int32_t width, int32_t height, const uint32_t* d_ranges,
                           const uint32_t* d_values, const float* d_xy, const float* d_conic_opacity,
                           const float* d_rgb, float* d_image, float* d_t_final, int32_t* d_n_contrib) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (width < 1 || height < 1 || width > 8192 || height > 8192 || !d_ranges || !d_xy || !d_conic_opacity ||
      !d_rgb || !d_image)
    return fail(c, FS4D_ERR_INVALID_ARG, "composite: bad argument");
  DeviceGuard g(c->device);
  FS4D_CUDA(c, launch_composite(width, height, reinterpret_cast<const uint2*>(d_ranges), d_values,
                                reinterpret_cast<const float2*>(d_xy), reinterpret_cast<const float4*>(d_conic_opacity),
                                d_rgb, d_image, d_t_final, d_n_contrib, c->stream));
  return FS4D_OK;
}

}  // extern "C"

// ============================================================== serving
// Continuous batching: a scheduler thread admits queued requests into work
// slots (each with its own stream, work memory and cached CUDA graphs) while
// device memory allows, deforms the admitted requests of one scene in one
// launch, and retires slots as their completion events fire.

namespace {

struct SReq {
  uint64_t ticket = 0;
  fs4d_request r{};
  double submit_ms = 0;
  long long pairs_hint = 0;
  int retries = 0;
};

struct GraphKey {
  int scene, w, h, prec;
  long long cap;
  bool operator<(const GraphKey& o) const {
    return std::tie(scene, w, h, prec, cap) < std::tie(o.scene, o.w, o.h, o.prec, o.cap);
  }
};

struct Slot {
  int id = 0;
  Work w;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  DevBuf status, dcam, dt, image;
  fs4d_camera* h_cam = nullptr;  // pinned staging
  float* h_t = nullptr;
  uint32_t* h_out = nullptr;     // [0] status word, [1] tile pairs
  int cap_w = 0, cap_h = 0;
  size_t bytes = 0;
  bool busy = false;
  SReq req;
  double start_ms = 0;
  Scene* scene = nullptr;
  std::map<GraphKey, cudaGraphExec_t> graphs;
};

struct Staging {
  DevBuf ts, tab;
  float* h_ts = nullptr;
  float** h_tab = nullptr;
  cudaEvent_t used = nullptr;
};

size_t slot_bytes_for(int n, int w, int h, long long pairs) {
  const size_t tiles = (size_t)tiles_of(w) * tiles_of(h);
  const size_t bmp = bitmap_bytes(n, (long long)tiles);
  return (bmp <= kBitmapMaxBytes ? bmp + 36 * (size_t)n : 0) + (size_t)n * (12 + 16 + 12 + 8 + 16 + 12 + 4 + 4 + 16 + 4 + 24) + 8 * (size_t)(emit_parts(n) + 1) +
         (size_t)pairs * 24 + 4 * 256 * (size_t)kSortMaxPasses * sort_parts(pairs) + tiles * 8 +
         (size_t)w * h * 12 + 4096;
}

}  // namespace

struct fs4d_server {
  fs4d_ctx* c = nullptr;
  fs4d_server_config cfg{};
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::deque<SReq> pending;
  std::vector<fs4d_completion> done;
  std::vector<Slot*> slots;
  uint64_t next_ticket = 1;
  std::chrono::steady_clock::time_point t0;
  cudaStream_t dstream = nullptr;
  DevBuf dstatus;  // status word of the batched deformation launches
  std::vector<Staging> staging;
  int staging_next = 0;
  std::map<std::tuple<int, int, int>, double> ppg;  // observed pairs per Gaussian per (scene, w, h)
  fs4d_server_stats stats{};
  int busy = 0;
  double now() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

void complete(fs4d_server* sv, const SReq& q, int32_t status, int slot, long long pairs, double start_ms) {
  fs4d_completion d{};
  d.ticket = q.ticket;
  d.status = status;
  d.slot = slot;
  d.pairs = pairs;
  d.submit_ms = q.submit_ms;
  d.start_ms = start_ms;
  d.done_ms = sv->now();
  std::lock_guard<std::mutex> lock(sv->mu);
  sv->done.push_back(d);
  if (status == FS4D_OK)
    sv->stats.completed++;
  else
    sv->stats.failed++;
  sv->cv.notify_all();
}

// Retire finished slots; a frame that overflowed its pair capacity is queued again.
void poll_slots(fs4d_server* sv) {
  for (Slot* sl : sv->slots) {
    if (!sl->busy) continue;
    const cudaError_t e = cudaEventQuery(sl->done);
    if (e == cudaErrorNotReady) continue;
    const uint32_t st = sl->h_out[0];
    const long long K = sl->h_out[1];
    sl->scene->refs--;
    sl->busy = false;
    const std::tuple<int, int, int> key{sl->req.r.scene, sl->req.r.cam.width, sl->req.r.cam.height};
    const double ratio = (double)K / std::max(1, sl->scene->n);
    if (e != cudaSuccess) {
      complete(sv, sl->req, FS4D_ERR_CUDA, sl->id, K, sl->start_ms);
    } else if (st & kStatusCapacity) {
      SReq q = sl->req;
      q.retries++;
      q.pairs_hint = std::max<long long>(K + K / 4, 2 * sl->w.cap_pairs);
      {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->ppg[key] = std::max(sv->ppg[key], ratio);
        sv->stats.retried++;
      }
      if (q.retries > 4) {
        complete(sv, q, FS4D_ERR_CAPACITY, sl->id, K, sl->start_ms);
      } else {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->pending.push_front(q);
      }
    } else if (st & kStatusTimeout) {
      complete(sv, sl->req, FS4D_ERR_TIMEOUT, sl->id, K, sl->start_ms);
    } else {
      {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->ppg[key] = std::max(sv->ppg[key], ratio);
      }
      complete(sv, sl->req, FS4D_OK, sl->id, K, sl->start_ms);
    }
    std::lock_guard<std::mutex> lock(sv->mu);  // after the completion or the re-queue: drain sees no gap
    sv->busy--;
  }
}

Slot* new_slot(fs4d_server* sv) {
  Slot* sl = new Slot();
  sl->id = (int)sv->slots.size();
  if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost(&sl->h_cam, sizeof(fs4d_camera)) != cudaSuccess ||
      cudaMallocHost(&sl->h_t, sizeof(float)) != cudaSuccess ||
      cudaMallocHost(&sl->h_out, 4 * sizeof(uint32_t)) != cudaSuccess || ensure(sl->status, 16) != cudaSuccess ||
      ensure(sl->dcam, sizeof(fs4d_camera)) != cudaSuccess || ensure(sl->dt, 16) != cudaSuccess) {
    return nullptr;  // (leaks a partly built slot only when the device is out of memory)
  }
  sv->slots.push_back(sl);
  return sl;
}

// Make the slot hold a frame of n Gaussians at w x h with `pairs` capacity.
fs4d_status fit_slot(fs4d_server* sv, Slot* sl, int n, int w, int h, long long pairs) {
  fs4d_ctx* c = sv->c;
  const void* before[6] = {sl->w.dmeans.p, sl->w.keys.p, sl->w.ranges.p, sl->w.zero.p, sl->image.p, sl->w.bitmap.p};
  fs4d_status st = ensure_work(c, sl->w, sl->stream, n, tiles_of(w) * tiles_of(h), pairs);
  if (st != FS4D_OK) return st;
  if ((size_t)w * h * 12 > sl->image.bytes) FS4D_CUDA(c, ensure(sl->image, (size_t)w * h * 12));
  const void* after[6] = {sl->w.dmeans.p, sl->w.keys.p, sl->w.ranges.p, sl->w.zero.p, sl->image.p, sl->w.bitmap.p};
  if (std::memcmp(before, after, sizeof(before)) != 0) {  // graphs captured on old buffers are stale
    cudaStreamSynchronize(sl->stream);
    for (auto& kv : sl->graphs) cudaGraphExecDestroy(kv.second);
    sl->graphs.clear();
  }
  sl->cap_w = std::max(sl->cap_w, w);
  sl->cap_h = std::max(sl->cap_h, h);
  const size_t b = slot_bytes_for(sl->w.cap_n, sl->cap_w, sl->cap_h, sl->w.cap_pairs);
  sv->stats.slot_bytes += (int64_t)b - (int64_t)sl->bytes;
  sl->bytes = b;
  sv->stats.peak_slot_bytes = std::max(sv->stats.peak_slot_bytes, sv->stats.slot_bytes);
  return FS4D_OK;
}

// The frame of one request, from its deformed Gaussians on, on the slot's stream
// (graph replay once captured for this scene/resolution/precision/capacity).
fs4d_status run_slot_frame(fs4d_server* sv, Slot* sl, Scene* s, const fs4d_request& r) {
  fs4d_ctx* c = sv->c;
  Env e{c, &sl->w, sl->stream, P<uint32_t>(sl->status), false};
  const long long cap = sl->w.cap_pairs;
  const GraphKey key{r.scene, r.cam.width, r.cam.height, (int)r.prec, cap};
  auto it = sl->graphs.find(key);
  if (it != sl->graphs.end()) {
    FS4D_CUDA(c, cudaGraphLaunch(it->second, sl->stream));
    return FS4D_OK;
  }
  // first frame of this kind on the slot: run it directly, then capture it
  const fs4d_camera* dcam = P<fs4d_camera>(sl->dcam);
  const float* dt = P<float>(sl->dt);
  float* img = P<float>(sl->image);
  fs4d_status st = frame_front(e, s, r.prec, r.cam, dcam, dt, 0.f, cap, true, false, false, true);
  if (st == FS4D_OK) st = frame_back(e, r.cam, cap, img, nullptr, nullptr, nullptr);
  if (st != FS4D_OK) return st;
  cudaGraph_t g = nullptr;
  FS4D_CUDA(c, cudaStreamBeginCapture(sl->stream, cudaStreamCaptureModeThreadLocal));
  fs4d_status st2 = frame_front(e, s, r.prec, r.cam, dcam, dt, 0.f, cap, true, false, false, true);
  if (st2 == FS4D_OK) st2 = frame_back(e, r.cam, cap, img, nullptr, nullptr, nullptr);
  const cudaError_t ce = cudaStreamEndCapture(sl->stream, &g);
  if (st2 != FS4D_OK) {
    if (g) cudaGraphDestroy(g);
    return st2;
  }
  FS4D_CUDA(c, ce);
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  FS4D_CUDA(c, ie);
  sl->graphs[key] = ex;
  return FS4D_OK;
}

// Admit a batch of queued requests that share the head request's scene and
// precision, as far as slots and the device-memory budget allow.
void admit_and_launch(fs4d_server* sv) {
  fs4d_ctx* c = sv->c;
  std::vector<std::pair<SReq, Slot*>> batch;
  Scene* scene = nullptr;
  {
    std::unique_lock<std::mutex> lock(sv->mu);
    if (sv->pending.empty()) return;
    const fs4d_scene_id sid = sv->pending.front().r.scene;
    const fs4d_precision prec = sv->pending.front().r.prec;
    bool unsupported = false;
    {
      std::lock_guard<std::mutex> cl(c->mu);
      auto it = c->scenes.find(sid);
      if (it != c->scenes.end() && !it->second->dying && !it->second->color_heads) {
        scene = it->second;
        scene->refs++;  // provisional: keeps the scene alive while the batch forms
      }
      unsupported = it != c->scenes.end() && it->second->color_heads;
    }
    if (!scene) {  // unknown, unloaded or unsupported scene: fail every queued request on it
      std::deque<SReq> keep;
      std::vector<SReq> bad;
      for (SReq& q : sv->pending) {
        if (q.r.scene == sid)
          bad.push_back(q);
        else
          keep.push_back(q);
      }
      sv->pending.swap(keep);
      lock.unlock();
      // the batched deformation of the server does not run the colour and opacity heads
      for (SReq& q : bad) complete(sv, q, unsupported ? FS4D_ERR_UNIMPLEMENTED : FS4D_ERR_NOT_FOUND, -1, 0, sv->now());
      return;
    }
    std::vector<bool> taken(sv->slots.size(), false);
    int64_t projected = sv->stats.slot_bytes;
    for (auto it = sv->pending.begin(); it != sv->pending.end() && (int)batch.size() < sv->cfg.max_batch;) {
      SReq& q = *it;
      if (q.r.scene != sid || q.r.prec != prec) {
        ++it;
        continue;
      }
      const auto key = std::make_tuple(q.r.scene, q.r.cam.width, q.r.cam.height);
      const double ratio = sv->ppg.count(key) ? sv->ppg[key] : (double)sv->cfg.pairs_per_gaussian;
      const long long want = std::max<long long>(q.pairs_hint, (long long)(1.3 * ratio * scene->n) + 4096);
      // a free slot that already fits, else a free slot to grow, else a new slot
      Slot* pick = nullptr;
      bool fits = false;
      for (size_t i = 0; i < sv->slots.size(); ++i) {
        Slot* sl = sv->slots[i];
        if (sl->busy || taken[i]) continue;
        if (sl->w.cap_n >= scene->n && sl->w.cap_pairs >= want && sl->cap_w >= q.r.cam.width &&
            sl->cap_h >= q.r.cam.height) {
          pick = sl;
          fits = true;
          break;
        }
        if (!pick) pick = sl;
      }
      if (!fits) {
        const size_t need = slot_bytes_for(std::max(scene->n, pick ? pick->w.cap_n : 0),
                                           std::max(q.r.cam.width, pick ? pick->cap_w : 0),
                                           std::max(q.r.cam.height, pick ? pick->cap_h : 0),
                                           std::max(want, pick ? pick->w.cap_pairs : 0));
        const int64_t have = pick ? (int64_t)pick->bytes : 0;
        const bool room = projected - have + (int64_t)need <= sv->cfg.hbm_budget_bytes;
        if (!room && batch.empty() && sv->busy == 0 && (int64_t)need > sv->cfg.hbm_budget_bytes) {
          SReq qq = q;  // can never fit: fail it instead of waiting forever
          sv->pending.erase(it);
          lock.unlock();
          complete(sv, qq, FS4D_ERR_OOM, -1, 0, sv->now());
          lock.lock();
          break;
        }
        if (!room) break;  // wait until device memory frees up
        if (!pick) {
          if ((int)sv->slots.size() >= sv->cfg.max_inflight) break;  // wait for a slot
          pick = new_slot(sv);
          if (!pick) break;
          taken.push_back(false);
        }
        projected += (int64_t)need - have;
      }
      taken[(size_t)pick->id] = true;
      batch.emplace_back(q, pick);
      it = sv->pending.erase(it);
    }
    scene->refs += (int)batch.size() - 1;  // the provisional reference becomes the batch's
    sv->busy += (int)batch.size();          // in flight from now on (drain waits for them)
  }
  if (batch.empty()) return;
  // grow the slots that need it (outside the queue lock)
  for (size_t i = 0; i < batch.size();) {
    const SReq& q = batch[i].first;
    Slot* sl = batch[i].second;
    const auto key = std::make_tuple(q.r.scene, q.r.cam.width, q.r.cam.height);
    double ratio;
    {
      std::lock_guard<std::mutex> lock(sv->mu);
      ratio = sv->ppg.count(key) ? sv->ppg[key] : (double)sv->cfg.pairs_per_gaussian;
    }
    const long long want = std::max<long long>(q.pairs_hint, (long long)(1.3 * ratio * scene->n) + 4096);
    if (fit_slot(sv, sl, scene->n, q.r.cam.width, q.r.cam.height, want) != FS4D_OK) {
      scene->refs--;
      {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->busy--;
      }
      complete(sv, q, FS4D_ERR_OOM, sl->id, 0, sv->now());
      batch.erase(batch.begin() + (long)i);
      continue;
    }
    ++i;
  }
  if (batch.empty()) return;
  // one deformation launch for the whole batch, written into each slot
  Staging& sg = sv->staging[(size_t)(sv->staging_next++ % (int)sv->staging.size())];
  cudaEventSynchronize(sg.used);
  const int nb = (int)batch.size();
  for (int i = 0; i < nb; ++i) {
    Slot* sl = batch[i].second;
    sg.h_ts[i] = batch[i].first.r.t;
    sg.h_tab[3 * i] = P<float>(sl->w.dmeans);
    sg.h_tab[3 * i + 1] = P<float>(sl->w.dquats);
    sg.h_tab[3 * i + 2] = P<float>(sl->w.dscales);
  }
  bool ok = cudaMemcpyAsync(sg.ts.p, sg.h_ts, 4 * (size_t)nb, cudaMemcpyHostToDevice, sv->dstream) == cudaSuccess &&
            cudaMemcpyAsync(sg.tab.p, sg.h_tab, 3 * sizeof(float*) * (size_t)nb, cudaMemcpyHostToDevice,
                            sv->dstream) == cudaSuccess;
  DeformArgs da = deform_args(scene, P<float>(sg.ts), 0.f, nb, nullptr, nullptr, nullptr);
  da.out_tab = P<float*>(sg.tab);
  const fs4d_precision prec = batch[0].first.r.prec;
  ok = ok && run_deform(c, scene, prec, da, sv->dstream, P<uint32_t>(sv->dstatus)) == FS4D_OK;
  ok = ok && cudaEventRecord(sg.used, sv->dstream) == cudaSuccess;
  sv->stats.batches++;
  sv->stats.deformed += nb;
  for (auto& bq : batch) {
    Slot* sl = bq.second;
    const fs4d_request& r = bq.first.r;
    sl->req = bq.first;
    sl->scene = scene;
    sl->start_ms = sv->now();
    *sl->h_cam = r.cam;
    *sl->h_t = r.t;
    bool sok = ok && cudaStreamWaitEvent(sl->stream, sg.used, 0) == cudaSuccess &&
               cudaMemcpyAsync(sl->dcam.p, sl->h_cam, sizeof(fs4d_camera), cudaMemcpyHostToDevice, sl->stream) ==
                   cudaSuccess &&
               cudaMemcpyAsync(sl->dt.p, sl->h_t, 4, cudaMemcpyHostToDevice, sl->stream) == cudaSuccess &&
               cudaMemsetAsync(sl->status.p, 0, 4, sl->stream) == cudaSuccess;
    sok = sok && run_slot_frame(sv, sl, scene, r) == FS4D_OK;
    const size_t bytes = (size_t)r.cam.width * r.cam.height * 12;
    sok = sok && cudaMemcpyAsync(r.out, sl->image.p, bytes,
                                 r.out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 sl->stream) == cudaSuccess;
    sok = sok && cudaMemcpyAsync(sl->h_out, sl->status.p, 4, cudaMemcpyDeviceToHost, sl->stream) == cudaSuccess &&
          cudaMemcpyAsync(sl->h_out + 1, sl->w.z.num_pairs, 4, cudaMemcpyDeviceToHost, sl->stream) == cudaSuccess &&
          cudaEventRecord(sl->done, sl->stream) == cudaSuccess;
    if (!sok) {
      scene->refs--;
      {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->busy--;
      }
      complete(sv, bq.first, FS4D_ERR_CUDA, sl->id, 0, sl->start_ms);
      continue;
    }
    sl->busy = true;
    int on_gpu = 0;
    for (Slot* x : sv->slots) on_gpu += x->busy ? 1 : 0;
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stats.max_concurrent = std::max(sv->stats.max_concurrent, on_gpu);
  }
}

void serve_loop(fs4d_server* sv) {
  cudaSetDevice(sv->c->device);
  for (;;) {
    poll_slots(sv);
    admit_and_launch(sv);
    std::unique_lock<std::mutex> lock(sv->mu);
    if (sv->stop && !sv->pending.empty()) {  // stopping: cancel what never started
      std::deque<SReq> q;
      q.swap(sv->pending);
      lock.unlock();
      for (SReq& r : q) complete(sv, r, FS4D_ERR_CANCELLED, -1, 0, sv->now());
      continue;
    }
    if (sv->stop && sv->busy == 0) break;
    sv->cv.notify_all();
    // sleep briefly: new work or a completion event will be there soon
    sv->cv.wait_for(lock, std::chrono::microseconds(sv->busy ? 20 : 200));
  }
}

}  // namespace

extern "C" {

fs4d_status fs4d_server_create(fs4d_ctx* c, const fs4d_server_config* cfg, fs4d_server** out) {
  if (!c || !cfg || !out) return FS4D_ERR_INVALID_ARG;
  if (cfg->max_inflight < 1 || cfg->max_batch < 1 || cfg->hbm_budget_bytes <= 0 || !(cfg->pairs_per_gaussian > 0))
    return fail(c, FS4D_ERR_INVALID_ARG, "server: max_inflight, max_batch, budget and pairs_per_gaussian > 0");
  if (c->server) return fail(c, FS4D_ERR_INVALID_ARG, "server: this context already has one");
  DeviceGuard g(c->device);
  fs4d_server* sv = new fs4d_server();
  sv->c = c;
  sv->cfg = *cfg;
  sv->t0 = std::chrono::steady_clock::now();
  if (cudaStreamCreateWithFlags(&sv->dstream, cudaStreamNonBlocking) != cudaSuccess ||
      ensure(sv->dstatus, 16) != cudaSuccess || cudaMemset(sv->dstatus.p, 0, 16) != cudaSuccess) {
    delete sv;
    return fail(c, FS4D_ERR_CUDA, "server: stream creation failed");
  }
  sv->staging.resize(8);
  for (Staging& s : sv->staging) {
    if (ensure(s.ts, 4 * (size_t)cfg->max_batch) != cudaSuccess ||
        ensure(s.tab, 3 * sizeof(float*) * (size_t)cfg->max_batch) != cudaSuccess ||
        cudaMallocHost(&s.h_ts, 4 * (size_t)cfg->max_batch) != cudaSuccess ||
        cudaMallocHost(&s.h_tab, 3 * sizeof(float*) * (size_t)cfg->max_batch) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.used, cudaEventDisableTiming) != cudaSuccess) {
      delete sv;
      return fail(c, FS4D_ERR_OOM, "server: staging allocation failed");
    }
  }
  c->server = sv;
  sv->th = std::thread(serve_loop, sv);
  *out = sv;
  return FS4D_OK;
}

fs4d_status fs4d_server_submit(fs4d_server* sv, const fs4d_request* r, uint64_t* ticket) {
  if (!sv || !r || !ticket) return FS4D_ERR_INVALID_ARG;
  if (!valid_cam(&r->cam) || !r->out || (r->prec != FS4D_FP32 && r->prec != FS4D_BF16)) return FS4D_ERR_INVALID_ARG;
  SReq q;
  q.r = *r;
  q.submit_ms = sv->now();
  std::lock_guard<std::mutex> lock(sv->mu);
  if (sv->stop) return FS4D_ERR_CANCELLED;
  q.ticket = sv->next_ticket++;
  *ticket = q.ticket;
  sv->pending.push_back(q);
  sv->stats.submitted++;
  sv->cv.notify_all();
  return FS4D_OK;
}

fs4d_status fs4d_server_submit_batch(fs4d_server* sv, const fs4d_request* reqs, int32_t n, uint64_t* tickets) {
  if (!sv || n < 0 || (n > 0 && (!reqs || !tickets))) return FS4D_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i)
    if (!valid_cam(&reqs[i].cam) || !reqs[i].out || (reqs[i].prec != FS4D_FP32 && reqs[i].prec != FS4D_BF16))
      return FS4D_ERR_INVALID_ARG;
  const double now = sv->now();
  std::lock_guard<std::mutex> lock(sv->mu);
  if (sv->stop) return FS4D_ERR_CANCELLED;
  for (int i = 0; i < n; ++i) {
    SReq q;
    q.r = reqs[i];
    q.submit_ms = now;
    q.ticket = sv->next_ticket++;
    tickets[i] = q.ticket;
    sv->pending.push_back(q);
  }
  sv->stats.submitted += n;
  sv->cv.notify_all();
  return FS4D_OK;
}

fs4d_status fs4d_server_cancel(fs4d_server* sv, uint64_t ticket) {
  if (!sv) return FS4D_ERR_INVALID_ARG;
  SReq q;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = std::find_if(sv->pending.begin(), sv->pending.end(), [&](const SReq& x) { return x.ticket == ticket; });
    if (it == sv->pending.end()) return FS4D_ERR_NOT_FOUND;
    q = *it;
    sv->pending.erase(it);
  }
  complete(sv, q, FS4D_ERR_CANCELLED, -1, 0, sv->now());
  return FS4D_OK;
}

fs4d_status fs4d_server_poll(fs4d_server* sv, fs4d_completion* out, int32_t max, int32_t* n_out) {
  if (!sv || !n_out || (max > 0 && !out)) return FS4D_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  const int n = std::min<int>(max, (int)sv->done.size());
  for (int i = 0; i < n; ++i) out[i] = sv->done[i];
  sv->done.erase(sv->done.begin(), sv->done.begin() + n);
  *n_out = n;
  return FS4D_OK;
}

fs4d_status fs4d_server_drain(fs4d_server* sv) {
  if (!sv) return FS4D_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lock(sv->mu);
  const bool ok = sv->cv.wait_for(lock, std::chrono::seconds(120), [&] { return sv->pending.empty() && sv->busy == 0; });
  return ok ? FS4D_OK : FS4D_ERR_TIMEOUT;
}

fs4d_status fs4d_server_stats_get(fs4d_server* sv, fs4d_server_stats* out) {
  if (!sv || !out) return FS4D_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(sv->mu);
  *out = sv->stats;
  out->slots = (int32_t)sv->slots.size();
  return FS4D_OK;
}

fs4d_status fs4d_server_destroy(fs4d_server* sv) {
  if (!sv) return FS4D_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stop = true;
    sv->cv.notify_all();
  }
  if (sv->th.joinable()) sv->th.join();
  fs4d_ctx* c = sv->c;
  DeviceGuard g(c->device);
  for (Slot* sl : sv->slots) {
    cudaStreamSynchronize(sl->stream);
    for (auto& kv : sl->graphs) cudaGraphExecDestroy(kv.second);
    Work& w = sl->w;
    DevBuf* all[] = {&w.dmeans, &w.dquats, &w.dscales, &w.xy, &w.co, &w.rgb, &w.depth, &w.radius, &w.rect,
                     &w.offsets, &w.emit_lb, &w.counters, &w.num_pairs, &w.hist, &w.keys, &w.values,
                     &w.keys_alt, &w.values_alt, &w.sort_lb, &w.ranges, &w.tile_count, &w.tile_order, &w.zero, &w.bitmap, &w.sxy, &w.sco, &w.srgb, &sl->status, &sl->dcam, &sl->dt,
                     &sl->image};
    for (DevBuf* b : all) release(*b);
    cudaFreeHost(sl->h_cam);
    cudaFreeHost(sl->h_t);
    cudaFreeHost(sl->h_out);
    cudaEventDestroy(sl->done);
    cudaStreamDestroy(sl->stream);
    delete sl;
  }
  cudaStreamSynchronize(sv->dstream);
  for (Staging& s : sv->staging) {
    release(s.ts);
    release(s.tab);
    if (s.h_ts) cudaFreeHost(s.h_ts);
    if (s.h_tab) cudaFreeHost(s.h_tab);
    if (s.used) cudaEventDestroy(s.used);
  }
  cudaStreamDestroy(sv->dstream);
  release(sv->dstatus);
  c->server = nullptr;
  delete sv;
  return FS4D_OK;
}

}  // extern "C"

// ============================================================== training step
// L = |I^ - I| + L_tv (Sec. 4.3) and one Adam update of every parameter group at
// learning rates decayed over the run (App. A), all on the device: render with the
// backward's state, L1 loss and dL/dI, backward, TV loss and its plane gradient,
// fused Adam (which also clears the gradients), refresh of the derived copies.

struct fs4d_trainer {
  fs4d_ctx* c = nullptr;
  fs4d_scene_id scene = 0;
  fs4d_train_config cfg{};
  long long step = 0;
  fs4d_frame frame;                          // reused from step to step
  DevBuf image, dl, partial, losses;         // [H][W][3] x 2, loss partials, [2] losses
  DevBuf grad, m, v;                         // every group, in the order of fs4d_scene_desc
  size_t off[7] = {}, count[7] = {};         // float offset and count of each group
  DevBuf stats;                              // densification statistics: [2][n] (gradient norm sum, views)
};

namespace {
void release_frame(fs4d_frame& f) {
  DevBuf* all[] = {&f.dmeans, &f.dquats, &f.dscales, &f.xy, &f.co, &f.rgb, &f.radius, &f.rect, &f.offsets,
                   &f.values, &f.ranges, &f.t_final, &f.n_contrib};
  for (DevBuf* b : all) release(*b);
}

double lr_at(const float lr[2], long long k, long long total) {
  if (total <= 0 || !(lr[0] > 0.f) || !(lr[1] > 0.f)) return lr[0];
  const double f = std::min(1.0, (double)k / (double)total);
  return std::exp((1.0 - f) * std::log((double)lr[0]) + f * std::log((double)lr[1]));
}
}  // namespace

extern "C" {

fs4d_status fs4d_train_create(fs4d_ctx* c, fs4d_scene_id id, const fs4d_train_config* cfg, fs4d_trainer** out) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (!cfg || !out) return fail(c, FS4D_ERR_INVALID_ARG, "train_create: config and output required");
  *out = nullptr;
  if (!(cfg->beta1 >= 0.f && cfg->beta1 < 1.f && cfg->beta2 >= 0.f && cfg->beta2 < 1.f && cfg->eps >= 0.f &&
        cfg->tv_weight >= 0.f && cfg->total_steps >= 0))
    return fail(c, FS4D_ERR_INVALID_ARG, "train_create: betas in [0,1), eps, tv_weight, total_steps >= 0");
  Scene* s;
  fs4d_status st = get_scene(c, id, &s);
  if (st != FS4D_OK) return st;
  if (s->color_heads)
    return fail(c, FS4D_ERR_UNIMPLEMENTED, "train_create: no backward through the colour and opacity heads");
  DeviceGuard g(c->device);
  fs4d_trainer* tr = new (std::nothrow) fs4d_trainer();
  if (!tr) return fail(c, FS4D_ERR_OOM, "train_create: allocation failed");
  tr->c = c;
  tr->scene = id;
  tr->cfg = *cfg;
  const size_t n = (size_t)s->n;
  const size_t cnt[7] = {3 * n, 3 * n, 4 * n, n, 3 * n * s->K, s->planes_floats, s->mlp_floats};
  size_t total = 0;
  for (int k = 0; k < 7; ++k) {
    tr->off[k] = total;
    tr->count[k] = cnt[k];
    total += (cnt[k] + 3) / 4 * 4;  // each group 16-byte aligned
  }
  const size_t parts = (size_t)train_partials();
  if (ensure(tr->grad, 4 * total) != cudaSuccess || ensure(tr->m, 4 * total) != cudaSuccess ||
      ensure(tr->v, 4 * total) != cudaSuccess || ensure(tr->partial, 4 * parts) != cudaSuccess ||
      ensure(tr->losses, 16) != cudaSuccess || ensure(tr->stats, 8 * n) != cudaSuccess) {
    fs4d_train_destroy(tr);
    return fail(c, FS4D_ERR_OOM, "train_create: device allocation failed");
  }
  if (cudaMemsetAsync(tr->grad.p, 0, 4 * total, c->stream) != cudaSuccess ||
      cudaMemsetAsync(tr->m.p, 0, 4 * total, c->stream) != cudaSuccess ||
      cudaMemsetAsync(tr->v.p, 0, 4 * total, c->stream) != cudaSuccess ||
      cudaMemsetAsync(tr->stats.p, 0, 8 * n, c->stream) != cudaSuccess) {
    fs4d_train_destroy(tr);
    return fail(c, FS4D_ERR_CUDA, "train_create: clearing the optimiser state failed");
  }
  *out = tr;
  return FS4D_OK;
}

fs4d_status fs4d_train_step(fs4d_trainer* tr, fs4d_precision prec, const fs4d_camera* cam, float t,
                            const float* d_target, float* d_losses) {
  NvtxScope nvtx_scope("fs4d:train_step");
  if (!tr) return FS4D_ERR_INVALID_ARG;
  fs4d_ctx* c = tr->c;
  if (!valid_cam(cam) || !d_target) return fail(c, FS4D_ERR_INVALID_ARG, "train_step: camera and target required");
  Scene* s;
  fs4d_status st = get_scene(c, tr->scene, &s);
  if (st != FS4D_OK) return st;
  if (tr->count[3] != (size_t)s->n)
    return fail(c, FS4D_ERR_INVALID_ARG, "train_step: the scene changed size without this trainer (densify with it)");
  DeviceGuard g(c->device);
  const size_t pix3 = 3 * (size_t)cam->width * cam->height;
  if (tr->image.bytes < 4 * pix3 || tr->dl.bytes < 4 * pix3) {
    FS4D_CUDA(c, cudaStreamSynchronize(c->stream));
    FS4D_CUDA(c, ensure(tr->image, 4 * pix3));
    FS4D_CUDA(c, ensure(tr->dl, 4 * pix3));
  }
  float* losses = d_losses ? d_losses : P<float>(tr->losses);
  // 1. the frame, keeping the backward's state
  if ((st = render_into_frame(c, s, prec, cam, t, P<float>(tr->image), &tr->frame)) != FS4D_OK) return st;
  // 2. L1 loss and dL/dI (misaligned targets take the scalar path inside the kernel)
  FS4D_CUDA(c, launch_l1(P<float>(tr->image), d_target, (long long)pix3, P<float>(tr->dl), P<float>(tr->partial),
                         losses, c->stream));
  // 3. backward into every group
  float* G = P<float>(tr->grad);
  fs4d_grads gr{G + tr->off[0], G + tr->off[1], G + tr->off[2], G + tr->off[3], G + tr->off[4], G + tr->off[5],
                G + tr->off[6]};
  const fs4d_view_stats vs{P<float>(tr->stats), P<float>(tr->stats) + s->n};
  if ((st = fs4d_render_backward_stats(c, &tr->frame, P<float>(tr->dl), &gr, &vs)) != FS4D_OK) return st;
  // 4. TV loss of the planes and its gradient
  FS4D_CUDA(c, launch_tv(s->pg, P<float>(s->planes), tr->cfg.tv_weight, gr.planes, P<float>(tr->partial), losses + 1,
                         c->stream));
  // 5. Adam at this step's learning rates
  const fs4d_train_config& q = tr->cfg;
  const long long k = tr->step, step = k + 1;
  AdamArgs a{};
  a.beta1 = q.beta1; a.beta2 = q.beta2; a.eps = q.eps;
  a.c1 = (float)(1.0 - std::pow((double)q.beta1, (double)step));
  a.c2 = (float)(1.0 - std::pow((double)q.beta2, (double)step));
  const float* lrs[7] = {q.lr_means, q.lr_log_scales, q.lr_quats, q.lr_opacity, q.lr_sh_rest, q.lr_planes, q.lr_mlp};
  DevBuf* params[7] = {&s->means, &s->log_scales, &s->quats, &s->opacity_logits, &s->sh, &s->planes, &s->mlp};
  for (int grp = 0; grp < 7; ++grp) {
    AdamSeg& sg = a.seg[a.n_segs++];
    sg.p = P<float>(*params[grp]);
    sg.g = G + tr->off[grp];
    sg.m = P<float>(tr->m) + tr->off[grp];
    sg.v = P<float>(tr->v) + tr->off[grp];
    sg.n = (long long)tr->count[grp];
    sg.lr = (float)lr_at(lrs[grp], k, q.total_steps);
    if (grp == 4) {  // SH: the degree-0 coefficients (3 of every 3K) take their own rate
      sg.period = 3 * s->K;
      sg.head = 3;
      sg.lr_head = (float)lr_at(q.lr_sh_dc, k, q.total_steps);
    }
    a.total += sg.n;
  }
  FS4D_CUDA(c, launch_adam(a, c->stream));
  // 6. the derived copies the next frame reads
  FS4D_CUDA(c, launch_derive(P<float>(s->planes), (long long)s->planes_floats, P<__nv_bfloat16>(s->planes_bf16),
                             P<float>(s->mlp), (int)s->mlp_floats, P<int4>(s->derive_tab), P<float>(s->mlp_t),
                             s->bf16_ok ? P<uint8_t>(s->tc_ops) : nullptr, s->bf16_ok ? P<float>(s->tc_bias) : nullptr,
                             c->stream));
  tr->step = step;
  return FS4D_OK;
}

fs4d_status fs4d_train_losses(fs4d_trainer* tr, float* h_losses) {
  if (!tr || !h_losses) return FS4D_ERR_INVALID_ARG;
  fs4d_ctx* c = tr->c;
  DeviceGuard g(c->device);
  FS4D_CUDA(c, cudaMemcpyAsync(h_losses, tr->losses.p, 8, cudaMemcpyDeviceToHost, c->stream));
  FS4D_CUDA(c, cudaStreamSynchronize(c->stream));
  return FS4D_OK;
}

fs4d_status fs4d_train_steps_done(const fs4d_trainer* tr, int64_t* steps) {
  if (!tr || !steps) return FS4D_ERR_INVALID_ARG;
  *steps = tr->step;
  return FS4D_OK;
}

fs4d_status fs4d_train_destroy(fs4d_trainer* tr) {
  if (!tr) return FS4D_OK;
  fs4d_ctx* c = tr->c;
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  release_frame(tr->frame);
  DevBuf* all[] = {&tr->image, &tr->dl, &tr->partial, &tr->losses, &tr->grad, &tr->m, &tr->v, &tr->stats};
  for (DevBuf* b : all) release(*b);
  delete tr;
  return FS4D_OK;
}

fs4d_status fs4d_train_read_state(fs4d_trainer* tr, int32_t group, float* h_m, float* h_v) {
  if (!tr) return FS4D_ERR_INVALID_ARG;
  fs4d_ctx* c = tr->c;
  if (group < 0 || group > 6) return fail(c, FS4D_ERR_INVALID_ARG, "train_read_state: group 0..6");
  DeviceGuard g(c->device);
  const size_t bytes = 4 * tr->count[group];
  if (h_m)
    FS4D_CUDA(c, cudaMemcpyAsync(h_m, P<float>(tr->m) + tr->off[group], bytes, cudaMemcpyDeviceToHost, c->stream));
  if (h_v)
    FS4D_CUDA(c, cudaMemcpyAsync(h_v, P<float>(tr->v) + tr->off[group], bytes, cudaMemcpyDeviceToHost, c->stream));
  FS4D_CUDA(c, cudaStreamSynchronize(c->stream));
  return FS4D_OK;
}

fs4d_status fs4d_train_stats(fs4d_trainer* tr, const fs4d_view_stats* out) {
  if (!tr || !out) return FS4D_ERR_INVALID_ARG;
  fs4d_ctx* c = tr->c;
  DeviceGuard g(c->device);
  const size_t n = tr->count[3];  // one opacity logit per Gaussian
  if (out->grad_norm_sum)
    FS4D_CUDA(c, cudaMemcpyAsync(out->grad_norm_sum, tr->stats.p, 4 * n, cudaMemcpyDeviceToDevice, c->stream));
  if (out->visible)
    FS4D_CUDA(c, cudaMemcpyAsync(out->visible, P<float>(tr->stats) + n, 4 * n, cudaMemcpyDeviceToDevice, c->stream));
  return FS4D_OK;
}

fs4d_status fs4d_densify(fs4d_ctx* c, fs4d_scene_id id, const fs4d_densify_config* cfg, const fs4d_view_stats* vs,
                         const float* d_normals, fs4d_trainer* tr, int64_t* n_out) {
  NvtxScope nvtx_scope("fs4d:densify");
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (!cfg || !vs || !vs->grad_norm_sum || !vs->visible || !d_normals || !n_out)
    return fail(c, FS4D_ERR_INVALID_ARG, "densify: config, statistics, normals and output required");
  Scene* s;
  fs4d_status st = get_scene(c, id, &s);
  if (st != FS4D_OK) return st;
  if (tr && (tr->c != c || tr->scene != id)) return fail(c, FS4D_ERR_INVALID_ARG, "densify: trainer of another scene");
  {
    std::lock_guard<std::mutex> lock(c->mu);
    if (s->refs.load() > 0) return fail(c, FS4D_ERR_CANCELLED, "densify: serving requests on this scene in flight");
    s->dying = true;  // no serving launch on the scene while it changes size
  }
  struct Restore {
    fs4d_ctx* c;
    Scene* s;
    ~Restore() {
      std::lock_guard<std::mutex> lock(c->mu);
      s->dying = false;
    }
  } restore{c, s};
  DeviceGuard g(c->device);
  const int n = s->n;
  const int K3 = 3 * s->K;
  const int nb = densify_blocks(n);
  DevBuf plan;  // block offsets [3][nb] and totals [3]
  auto cleanup = [](std::initializer_list<DevBuf*> bufs) {
    for (DevBuf* b : bufs) release(*b);
  };
  FS4D_CUDA(c, ensure(plan, 4 * (3 * (size_t)nb + 4)));
  DensifyArgs a{};
  a.n = n;
  a.log_scales = P<float>(s->log_scales);
  a.opacity = P<float>(s->opacity_logits);
  a.grad_sum = vs->grad_norm_sum;
  a.visible = vs->visible;
  a.grad_threshold = cfg->grad_threshold;
  a.split_log_scale = cfg->split_log_scale;
  a.prune_logit = cfg->prune_logit;
  a.block_off = P<uint32_t>(plan);
  a.totals = P<uint32_t>(plan) + 3 * (size_t)nb;
  uint32_t tot[3] = {0, 0, 0};
  cudaError_t e = launch_densify_plan(a, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tot, a.totals, 12, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    cleanup({&plan});
    return fail(c, FS4D_ERR_CUDA, std::string("densify: ") + cudaGetErrorString(e));
  }
  const long long m = (long long)tot[0] + tot[1] + 2LL * tot[2];
  if (m == 0) {
    cleanup({&plan});
    return fail(c, FS4D_ERR_INVALID_ARG, "densify: every Gaussian would be removed");
  }
  if (m >= (1LL << 30)) {
    cleanup({&plan});
    return fail(c, FS4D_ERR_CAPACITY, "densify: more than 2^30 - 1 Gaussians");
  }
  // the new arrays, the output map and the work order's sort buffers
  DevBuf map, nm, nls, nq, no, nsh, keys, perm;
  std::initializer_list<DevBuf*> fresh = {&map, &nm, &nls, &nq, &no, &nsh, &keys, &perm};
  if (ensure(map, 8 * (size_t)m) != cudaSuccess || ensure(nm, 12 * (size_t)m) != cudaSuccess ||
      ensure(nls, 12 * (size_t)m) != cudaSuccess || ensure(nq, 16 * (size_t)m) != cudaSuccess ||
      ensure(no, 4 * (size_t)m) != cudaSuccess || ensure(nsh, 4 * (size_t)K3 * m) != cudaSuccess ||
      ensure(keys, 8 * (size_t)m) != cudaSuccess || ensure(perm, 4 * (size_t)m) != cudaSuccess) {
    cleanup({&plan});
    cleanup(fresh);
    return fail(c, FS4D_ERR_OOM, "densify: device allocation failed");
  }
  a.src = P<int32_t>(map);
  a.kind = P<int32_t>(map) + m;
  e = launch_densify_map(a, c->stream);
  const float* olds[5] = {P<float>(s->means), P<float>(s->log_scales), P<float>(s->quats), P<float>(s->opacity_logits),
                          P<float>(s->sh)};
  float* news[5] = {P<float>(nm), P<float>(nls), P<float>(nq), P<float>(no), P<float>(nsh)};
  const int width[5] = {3, 3, 4, 1, K3};
  for (int k = 0; k < 5 && e == cudaSuccess; ++k)
    e = launch_gather(olds[k], news[k], a.src, a.kind, m, width[k], false, c->stream);
  if (e == cudaSuccess) {
    ChildArgs ca{};
    ca.first = (long long)tot[0] + tot[1];
    ca.end = m;
    ca.src = a.src;
    ca.kind = a.kind;
    ca.means = olds[0];
    ca.log_scales = olds[1];
    ca.quats = olds[2];
    ca.normals = d_normals;
    ca.out_means = news[0];
    ca.out_log_scales = news[1];
    e = launch_children(ca, c->stream);
  }
  if (e == cudaSuccess)
    e = launch_morton(news[0], (int)m, s->shape.aabb_min, s->shape.aabb_max, P<unsigned long long>(keys),
                      P<uint32_t>(perm), c->stream);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(c->stream);
    cleanup({&plan});
    cleanup(fresh);
    return fail(c, FS4D_ERR_CUDA, std::string("densify: ") + cudaGetErrorString(e));
  }
  // the deformation work order of the new set: stable sort by Morton code
  if ((st = fs4d_sort_pairs(c, m, 30, P<uint64_t>(keys), P<uint32_t>(perm))) != FS4D_OK) {
    cudaStreamSynchronize(c->stream);
    cleanup({&plan});
    cleanup(fresh);
    return st;
  }
  // the trainer's state follows the Gaussians
  DevBuf tg, tm, tv, ts;
  size_t toff[7] = {}, tcnt[7] = {};
  if (tr) {
    const size_t cnt[7] = {3 * (size_t)m, 3 * (size_t)m, 4 * (size_t)m, (size_t)m, (size_t)K3 * m, tr->count[5],
                           tr->count[6]};
    size_t total = 0;
    for (int k = 0; k < 7; ++k) {
      toff[k] = total;
      tcnt[k] = cnt[k];
      total += (cnt[k] + 3) / 4 * 4;
    }
    if (ensure(tg, 4 * total) != cudaSuccess || ensure(tm, 4 * total) != cudaSuccess ||
        ensure(tv, 4 * total) != cudaSuccess || ensure(ts, 8 * (size_t)m) != cudaSuccess) {
      cudaStreamSynchronize(c->stream);
      cleanup({&plan, &tg, &tm, &tv, &ts});
      cleanup(fresh);
      return fail(c, FS4D_ERR_OOM, "densify: device allocation of the optimiser state failed");
    }
    e = cudaMemsetAsync(tg.p, 0, 4 * total, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ts.p, 0, 8 * (size_t)m, c->stream);
    for (int k = 0; k < 7 && e == cudaSuccess; ++k) {
      DevBuf* src[2] = {&tr->m, &tr->v};
      DevBuf* dst[2] = {&tm, &tv};
      for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
        const float* from = P<float>(*src[q]) + tr->off[k];
        float* to = P<float>(*dst[q]) + toff[k];
        if (k < 5)
          e = launch_gather(from, to, a.src, a.kind, m, width[k], true, c->stream);
        else
          e = cudaMemcpyAsync(to, from, 4 * tcnt[k], cudaMemcpyDeviceToDevice, c->stream);
      }
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaStreamSynchronize(c->stream);
    cleanup({&plan, &tg, &tm, &tv, &ts});
    cleanup(fresh);
    return fail(c, FS4D_ERR_CUDA, std::string("densify: ") + cudaGetErrorString(e));
  }
  // swap the new arrays in; the old ones are released with the temporaries
  const size_t per = 4 * (3 + 3 + 4 + 1 + (size_t)K3 + 1);
  std::swap(s->means, nm);
  std::swap(s->log_scales, nls);
  std::swap(s->quats, nq);
  std::swap(s->opacity_logits, no);
  std::swap(s->sh, nsh);
  std::swap(s->perm, perm);
  s->resident = s->resident - per * (size_t)n + per * (size_t)m;
  s->n = (int)m;
  s->shape.n = (int32_t)m;
  s->reserved_pairs = 0;
  s->reserved_w = s->reserved_h = 0;
  if (tr) {
    std::swap(tr->grad, tg);
    std::swap(tr->m, tm);
    std::swap(tr->v, tv);
    std::swap(tr->stats, ts);
    for (int k = 0; k < 7; ++k) {
      tr->off[k] = toff[k];
      tr->count[k] = tcnt[k];
    }
  }
  cleanup({&plan, &tg, &tm, &tv, &ts});
  cleanup(fresh);
  *n_out = m;
  return FS4D_OK;
}

fs4d_status fs4d_train_densify(fs4d_trainer* tr, const fs4d_densify_config* cfg, const float* d_normals,
                               int64_t* n_out) {
  if (!tr) return FS4D_ERR_INVALID_ARG;
  const fs4d_view_stats vs{P<float>(tr->stats), P<float>(tr->stats) + tr->count[3]};
  return fs4d_densify(tr->c, tr->scene, cfg, &vs, d_normals, tr, n_out);
}

}  // extern "C"

// ============================================================== scene read-back and files
namespace {
constexpr char kSceneMagic[8] = {'F', 'S', '4', 'D', 'S', 'C', 'N', '2'};    // 11 int32
constexpr char kSceneMagicV1[8] = {'F', 'S', '4', 'D', 'S', 'C', 'N', '1'};  // 10 int32, no color_heads

uint64_t fnv1a(uint64_t h, const void* p, size_t bytes) {
  const unsigned char* b = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < bytes; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

void group_sizes(const Scene* s, size_t cnt[7]) {
  const size_t n = (size_t)s->n;
  const size_t c[7] = {3 * n, 3 * n, 4 * n, n, 3 * n * s->K, s->planes_floats, s->mlp_floats};
  for (int k = 0; k < 7; ++k) cnt[k] = c[k];
}
}  // namespace

extern "C" {

fs4d_status fs4d_read_scene(fs4d_ctx* c, fs4d_scene_id id, const fs4d_grads* out, int32_t to_device) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (!out) return fail(c, FS4D_ERR_INVALID_ARG, "read_scene: output pointers required");
  Scene* s;
  fs4d_status st = get_scene(c, id, &s);
  if (st != FS4D_OK) return st;
  DeviceGuard g(c->device);
  size_t cnt[7];
  group_sizes(s, cnt);
  float* dst[7] = {out->means, out->log_scales, out->quats, out->opacity_logits, out->sh, out->planes, out->mlp};
  const DevBuf* src[7] = {&s->means, &s->log_scales, &s->quats, &s->opacity_logits, &s->sh, &s->planes, &s->mlp};
  const cudaMemcpyKind kind = to_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int k = 0; k < 7; ++k) {
    if (!dst[k]) continue;
    FS4D_CUDA(c, cudaMemcpyAsync(dst[k], src[k]->p, 4 * cnt[k], kind, c->stream));
  }
  FS4D_CUDA(c, cudaStreamSynchronize(c->stream));
  return FS4D_OK;
}

fs4d_status fs4d_save_scene(fs4d_ctx* c, fs4d_scene_id id, const char* path) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (!path) return fail(c, FS4D_ERR_INVALID_ARG, "save_scene: path required");
  Scene* s;
  fs4d_status st = get_scene(c, id, &s);
  if (st != FS4D_OK) return st;
  size_t cnt[7];
  group_sizes(s, cnt);
  std::vector<std::vector<float>> host(7);
  for (int k = 0; k < 7; ++k) host[k].resize(cnt[k]);
  fs4d_grads out{host[0].data(), host[1].data(), host[2].data(), host[3].data(), host[4].data(), host[5].data(),
                 host[6].data()};
  if ((st = fs4d_read_scene(c, id, &out, 0)) != FS4D_OK) return st;
  const fs4d_scene_desc& d = s->shape;
  const int32_t ints[11] = {d.n, d.sh_degree, d.n_levels, d.res_spatial[0], d.res_spatial[1], d.res_spatial[2],
                            d.res_spatial[3], d.res_time, d.feat_dim, d.mlp_width, d.color_heads};
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return fail(c, FS4D_ERR_INVALID_ARG, "save_scene: cannot open " + tmp);
  uint64_t h = 14695981039346656037ull;
  bool ok = std::fwrite(kSceneMagic, 1, 8, f) == 8;
  auto put = [&](const void* p, size_t bytes) {
    ok = ok && std::fwrite(p, 1, bytes, f) == bytes;
    h = fnv1a(h, p, bytes);
  };
  put(ints, sizeof(ints));
  put(d.aabb_min, sizeof(d.aabb_min));
  put(d.aabb_max, sizeof(d.aabb_max));
  for (int k = 0; k < 7; ++k) put(host[k].data(), 4 * cnt[k]);
  ok = ok && std::fwrite(&h, 1, 8, f) == 8;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return fail(c, FS4D_ERR_INVALID_ARG, std::string("save_scene: writing ") + path + " failed");
  }
  return FS4D_OK;
}

fs4d_status fs4d_load_scene_file(fs4d_ctx* c, const char* path, fs4d_scene_id* out) {
  if (!c) return FS4D_ERR_INVALID_ARG;
  if (!path || !out) return fail(c, FS4D_ERR_INVALID_ARG, "load_scene_file: path and output required");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(c, FS4D_ERR_NOT_FOUND, std::string("load_scene_file: cannot open ") + path);
  char magic[8];
  int32_t ints[11] = {};
  fs4d_scene_desc d{};
  uint64_t h = 14695981039346656037ull;
  bool ok = std::fread(magic, 1, 8, f) == 8;
  const bool v1 = ok && std::memcmp(magic, kSceneMagicV1, 8) == 0;
  ok = ok && (v1 || std::memcmp(magic, kSceneMagic, 8) == 0);
  auto get = [&](void* p, size_t bytes) {
    ok = ok && std::fread(p, 1, bytes, f) == bytes;
    if (ok) h = fnv1a(h, p, bytes);
  };
  get(ints, v1 ? 10 * sizeof(int32_t) : sizeof(ints));
  get(d.aabb_min, sizeof(d.aabb_min));
  get(d.aabb_max, sizeof(d.aabb_max));
  d.n = ints[0]; d.sh_degree = ints[1]; d.n_levels = ints[2];
  for (int l = 0; l < 4; ++l) d.res_spatial[l] = ints[3 + l];
  d.res_time = ints[7]; d.feat_dim = ints[8]; d.mlp_width = ints[9]; d.color_heads = ints[10];
  ok = ok && d.n >= 1 && d.sh_degree >= 0 && d.sh_degree <= 3 && d.n_levels >= 1 && d.n_levels <= kMaxLevels &&
       d.feat_dim > 0 && d.res_time >= 2 && d.mlp_width == kWidth && (d.color_heads == 0 || d.color_heads == 1);
  std::vector<std::vector<float>> host(7);
  if (ok) {
    PlaneGeom pg{};
    size_t planes_total = 0, mlp_total = 0;
    plane_geom(d, pg, planes_total);
    mlp_total = mlp_floats_of(d);
    const size_t n = (size_t)d.n, K = (size_t)(d.sh_degree + 1) * (d.sh_degree + 1);
    const size_t cnt[7] = {3 * n, 3 * n, 4 * n, n, 3 * n * K, planes_total, mlp_total};
    for (int k = 0; k < 7 && ok; ++k) {
      host[k].resize(cnt[k]);
      get(host[k].data(), 4 * cnt[k]);
    }
  }
  uint64_t stored = 0;
  ok = ok && std::fread(&stored, 1, 8, f) == 8 && stored == h;
  std::fclose(f);
  if (!ok) return fail(c, FS4D_ERR_INVALID_ARG, std::string("load_scene_file: ") + path + " is not a valid scene file");
  d.means = host[0].data(); d.log_scales = host[1].data(); d.quats = host[2].data();
  d.opacity_logits = host[3].data(); d.sh = host[4].data(); d.planes = host[5].data(); d.mlp = host[6].data();
  return fs4d_load_scene(c, &d, out);
}

}  // extern "C"
