// Tile binning: the per-tile lists of Gaussians in (depth, index) order, from the
// depth-sorted Gaussians and their tile rectangles, by one of two routes.
//
// Key emission (then a stable radix sort on the tile bits): one (tile | depth) key
// per (Gaussian, touched tile).  Gaussians are visited in a given order (the depth-sorted order, so that a
// stable sort on the tile bits alone yields (tile, depth, index) order).  One
// pass per 256-Gaussian partition:
//   1. exclusive scan of the tile counts, chained across CTAs by decoupled
//      look-back (partition index from an atomic ticket, so every predecessor a
//      CTA waits on is already resident; bounded spin);
//   2. cooperative emission: the CTA's pairs [0, total) are produced by
//      consecutive threads -- each finds its Gaussian by binary search over the
//      CTA's offsets in shared memory -- so key/value stores are coalesced;
//   3. per-tile pair counts in shared memory, merged by one global atomic per
//      non-empty tile.
// A one-CTA kernel scans the tile counts into the tile [start, end) ranges and
// the digit histograms of the pair sort that follows (no pass over the keys).
//
// Tile bitmap (no pair sort): one bit per (tile, depth rank), set by mark_kernel;
// after the same tile scan, extract_kernel reads each tile's row in rank order
// into the tile's range (see the tile bitmap section below).
#include "sync_util.cuh"

namespace fs4d {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 1;
constexpr int kPart = kThreads * kItems;  // Gaussians per partition
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr int kMaxPasses = 8;
constexpr int kEmitSmemTiles = 16384;     // tiles counted in shared memory (more: global atomics)

__global__ void __launch_bounds__(kThreads) scan_emit_kernel(EmitArgs a, int smem_tiles) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ uint32_t s_tc[];      // per-tile pair counts of this partition (smem_tiles != 0)
  __shared__ uint32_t s_part;
  __shared__ uint32_t s_warp[kThreads / 32];
  __shared__ unsigned long long s_prefix;
  __shared__ uint32_t s_off[kPart + 1];   // local exclusive offsets; s_off[kPart] = partition total
  __shared__ int4 s_rect[kPart];
  __shared__ uint32_t s_dbits[kPart];
  __shared__ uint32_t s_gid[kPart];
  const int tid = threadIdx.x;
  if (tid == 0) s_part = atomicAdd(a.part_counter, 1u);
  for (int i = tid; i < smem_tiles; i += kThreads) s_tc[i] = 0;
  __syncthreads();
  const int part = (int)s_part;
  const int base = part * kPart;
  const uint32_t* order = (a.order_sel && *a.order_sel) ? a.order_alt : a.order;

  // ---- 1. counts and the partition-local scan (thread t owns item t)
  uint32_t cnt[kItems];
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int li = tid * kItems + i;
    const int pos = base + li;
    cnt[i] = 0;
    int4 r = make_int4(0, 0, 0, 0);
    uint32_t g = 0, db = 0;
    if (pos < a.n) {
      g = order ? order[pos] : (uint32_t)pos;
      r = a.rect[g];
      db = __float_as_uint(a.depth[g]);
      cnt[i] = (uint32_t)max(0, r.z - r.x) * (uint32_t)max(0, r.w - r.y);
    }
    s_rect[li] = r;
    s_dbits[li] = db;
    s_gid[li] = g;
    sum += cnt[i];
  }
  const uint32_t lane = lane_id(), warp = tid / 32;
  uint32_t incl = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= (uint32_t)d) incl += v;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  uint32_t warp_excl = 0, block_total = 0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) {
    const uint32_t v = s_warp[w];
    if ((uint32_t)w < warp) warp_excl += v;
    block_total += v;
  }
  uint32_t run = warp_excl + incl - sum;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    s_off[tid * kItems + i] = run;
    run += cnt[i];
  }
  if (tid == 0) s_off[kPart] = block_total;

  // ---- chain the partitions
  if (tid == 0) {
    unsigned long long prefix = 0;
    if (part == 0) {
      st_relaxed_u64(&a.lookback[0], kFlagInc | block_total);
    } else {
      st_relaxed_u64(&a.lookback[part], kFlagAgg | block_total);
      // windowed look-back: 8 predecessors per round of independent loads
      constexpr int kWin = 8;
      int j = part - 1;
      uint32_t spins = 0;
      bool found = false;
      while (j >= 0 && !found) {
        const int cnt = min(kWin, j + 1);
        unsigned long long wv[kWin];
#pragma unroll
        for (int i = 0; i < kWin; ++i)
          if (i < cnt) wv[i] = ld_relaxed_u64(&a.lookback[j - i]);
        int used = 0;
#pragma unroll
        for (int i = 0; i < kWin; ++i) {
          if (i >= cnt || found) break;
          const unsigned long long flag = wv[i] & ~kValMask;
          if (flag == 0) break;
          prefix += wv[i] & kValMask;
          ++used;
          if (flag == kFlagInc) found = true;
        }
        j -= used;
        if (!found && used < cnt) {
          if (++spins > a.spin_limit) {
            atomicOr(a.status, kStatusTimeout);
            break;
          }
          __nanosleep(32);
        }
      }
      st_relaxed_u64(&a.lookback[part], kFlagInc | (prefix + block_total));
    }
    s_prefix = prefix;
    if ((long long)(part + 1) * kPart >= a.n) {
      const unsigned long long K = prefix + block_total;
      *a.num_pairs = K > 0xffffffffull ? 0xffffffffu : (uint32_t)K;
      const bool fits = (long long)K <= a.capacity;
      *a.num_pairs_sort = fits ? (uint32_t)K : 0u;
      if (!fits && a.report_overflow) atomicOr(a.status, kStatusCapacity);
    }
  }
  __syncthreads();
  const unsigned long long prefix = s_prefix;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int pos = base + tid * kItems + i;
    if (pos < a.n) a.offsets[s_gid[tid * kItems + i]] = (uint32_t)(prefix + s_off[tid * kItems + i]);
  }

  // ---- 2. cooperative emission, 3. per-tile pair counts
  for (uint32_t j0 = 0; j0 < block_total; j0 += kThreads) {
    const uint32_t j = j0 + (uint32_t)tid;
    const bool valid = j < block_total;
    unsigned long long key = 0;
    if (valid) {
      int lo = 0, hi = kPart - 1;  // last li with s_off[li] <= j; a Gaussian with no tiles never wins
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_off[mid] <= j)
          lo = mid;
        else
          hi = mid - 1;
      }
      const int4 r = s_rect[lo];
      const uint32_t k = j - s_off[lo];
      const uint32_t w = (uint32_t)(r.z - r.x);
      const uint32_t tile = (uint32_t)(r.y + (int)(k / w)) * (uint32_t)a.tiles_x + (uint32_t)(r.x + (int)(k % w));
      const unsigned long long out = prefix + j;
      if (a.packed) {  // (tile | Gaussian index): the sort carries the index in the key
        if ((long long)out < a.capacity) a.keys[out] = ((unsigned long long)tile << 32) | s_gid[lo];
      } else {
        key = ((unsigned long long)tile << 32) | s_dbits[lo];
        if ((long long)out < a.capacity) {
          a.keys[out] = key;
          a.values[out] = s_gid[lo];
        }
      }
      if (smem_tiles)
        atomicAdd(&s_tc[tile], 1u);
      else
        atomicAdd(&a.tile_count[tile], 1u);
    }
  }
  if (smem_tiles) {
    __syncthreads();
    for (int t = tid; t < smem_tiles; t += kThreads) {
      const uint32_t v = s_tc[t];
      if (v) atomicAdd(&a.tile_count[t], v);
    }
  }
}

// One CTA: exclusive scan of the per-tile pair counts.  A stable sort of the
// pairs on their tile bits puts tile t at [scan(t), scan(t) + count(t)), so this
// IS the tile range table (0, 0 for an empty tile, and for every tile when the
// pairs overflowed the buffers); the digit histograms of the pair sort's passes
// (digit p of tile t is (t >> 8p) & 255) come from the same counts.
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) tile_scan_kernel(const uint32_t* __restrict__ tile_count, int n_tiles,
                                                                 uint32_t* __restrict__ num_pairs,
                                                                 uint2* __restrict__ ranges, uint32_t* __restrict__ hist,
                                                                 int passes, uint32_t* __restrict__ order,
                                                                 long long capacity, uint32_t* __restrict__ status) {
  __shared__ uint32_t s_warp[kScanThreads / 32];
  __shared__ uint32_t s_hist[kMaxPasses][256];
  __shared__ uint32_t s_len[33];          // tiles per length class floor(log2(count)) + 1 (0: empty)
  pdl_wait();
  pdl_trigger();
  const int tid = threadIdx.x;
  const uint32_t lane = lane_id(), warp = tid / 32;
  for (int i = tid; i < kMaxPasses * 256; i += kScanThreads) (&s_hist[0][0])[i] = 0;
  if (tid < 33) s_len[tid] = 0;
  const bool sort_overflow = capacity < 0 && num_pairs[1] == 0u && num_pairs[0] != 0u;
  const int per = (n_tiles + kScanThreads - 1) / kScanThreads;
  const int t0 = min(tid * per, n_tiles), t1 = min(t0 + per, n_tiles);
  uint32_t sum = 0;
  for (int t = t0; t < t1; ++t) sum += tile_count[t];
  uint32_t incl = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= (uint32_t)d) incl += v;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  uint32_t run = incl - sum;
  unsigned long long total = 0;
  for (int w = 0; w < kScanThreads / 32; ++w) {
    if (w < (int)warp) run += s_warp[w];
    total += s_warp[w];
  }
  const bool overflow = capacity < 0 ? sort_overflow : (long long)total > capacity;
  if (capacity >= 0 && tid == 0) {
    num_pairs[1] = overflow ? 0u : (uint32_t)total;
    if (overflow && status) atomicOr(status, kStatusCapacity);
  }
  for (int t = t0; t < t1; ++t) {
    const uint32_t c = tile_count[t];
    if (ranges) ranges[t] = (overflow || c == 0) ? make_uint2(0u, 0u) : make_uint2(run, run + c);
    if (c && hist)
      for (int p = 0; p < passes; ++p) atomicAdd(&s_hist[p][((uint32_t)t >> (8 * p)) & 255u], c);
    run += c;
  }
  if (hist) {
    __syncthreads();
    for (int i = tid; i < passes * 256; i += kScanThreads) hist[i] = (&s_hist[0][0])[i];
  }
  if (order) {
    // Launch order for the compositing: tiles by length class, longest first, so
    // the longest lists start first and do not form the tail.  Tiles of one class
    // within a warp share one shared-memory atomic (most tiles of a frame are in
    // a few classes, empty ones above all).
    const uint32_t lane_lt = (1u << lane) - 1u;
    for (int b = 0; b < n_tiles; b += kScanThreads) {
      const int t = b + tid;
      const uint32_t c = (t < n_tiles && !overflow) ? tile_count[t] : 0u;
      const int cls = t < n_tiles ? 32 - (c ? 32 - __clz(c) : 0) : 33;
      const uint32_t peers = __match_any_sync(0xffffffffu, cls);
      if (cls < 33 && (peers & lane_lt) == 0) atomicAdd(&s_len[cls], (uint32_t)__popc(peers));
    }
    __syncthreads();
    if (tid == 0) {
      uint32_t run2 = 0;
      for (int b = 0; b < 33; ++b) {
        const uint32_t v = s_len[b];
        s_len[b] = run2;
        run2 += v;
      }
    }
    __syncthreads();
    for (int b = 0; b < n_tiles; b += kScanThreads) {
      const int t = b + tid;
      const uint32_t c = (t < n_tiles && !overflow) ? tile_count[t] : 0u;
      const int cls = t < n_tiles ? 32 - (c ? 32 - __clz(c) : 0) : 33;
      const uint32_t peers = __match_any_sync(0xffffffffu, cls);
      const int leader = __ffs(peers) - 1;
      uint32_t at = 0;
      if (cls < 33 && lane == (uint32_t)leader) at = atomicAdd(&s_len[cls], (uint32_t)__popc(peers));
      at = __shfl_sync(0xffffffffu, at, leader);
      if (cls < 33) order[at + __popc(peers & lane_lt)] = (uint32_t)t;
    }
  }
}

// ------------------------------------------------------------ tile bitmap
// The alternative to emission + pair sort: a bitmap with one row per tile and one
// bit per depth rank.  Row t read in rank order lists tile t's Gaussians in
// (depth, index) order -- exactly the order a stable sort of (tile | depth) keys
// gives -- so no sort is needed once the bits are set.

// Row r, column k - r * w of the k-th tile of a w-wide rectangle (row-major):
// the quotient from a float reciprocal, corrected by one step (exact for k < 2^22,
// where the float estimate is off by less than one); integer division above.
__device__ __forceinline__ uint32_t rect_row(uint32_t k, uint32_t w) {
  if (k >= (1u << 22)) return k / w;
  int r = __float2int_rz(((float)k + 0.5f) * __frcp_rn((float)w));
  const int c = (int)k - r * (int)w;
  r += c < 0 ? -1 : (c >= (int)w ? 1 : 0);
  return (uint32_t)r;
}

// 256 consecutive depth ranks per CTA; warps w and w + 8 own ranks [32w, 32w + 32)
// of the CTA, i.e. one word column of every row, and each takes every other chunk
// of 32 of the column's pairs (half the chain of dependent steps per warp).  A
// warp spreads a chunk over its lanes (binary search over the column's exclusive
// pair offsets by shuffles), and each pair sets its bit with one global atomic OR.
// Pairs per tile are summed in shared memory and merged by one global atomic per
// touched tile.  A rank's projected Gaussian is copied to its rank's slot when
// sorted copies are asked for.
constexpr int kMarkHalves = 2;  // warps per word column: each takes every other 32-pair chunk
constexpr int kMarkThreads = kPart * kMarkHalves;

// The ellipse {alpha >= 1/255} of a projected Gaussian for the tile test of culled
// lists: (A, B, C) its conic, S the bound on d^T K d wherever alpha may reach 1/255
// (a 0.4% + 2e-3 margin over the compositing's own), (kx, ky) the edge minimisers'
// slopes, (px, py) the mean.  S < 0: alpha never reaches 1/255; S = kNoBound: no
// usable bound (not positive definite), every tile of the rectangle is kept.
constexpr float kNoBound = 3.0e38f;
struct TileEllipse {
  float A, B, C, S, kx, ky, px, py;
};
__device__ __forceinline__ TileEllipse tile_ellipse(float2 p, float4 co) {
  TileEllipse e{co.x, co.y, co.z, -1.f, 0.f, 0.f, p.x, p.y};
  const float thr = composite_exp_threshold(co.w);
  if (!(thr < 0.f)) return e;
  if (!(e.A > 0.f && e.C > 0.f && e.A * e.C - e.B * e.B > 0.f)) {
    e.S = kNoBound;
    return e;
  }
  e.S = -2.f * thr * 1.004f + 2e-3f;
  e.kx = -e.B / e.C;
  e.ky = -e.B / e.A;
  return e;
}
// Whether some pixel centre of tile (tx, ty) may blend the Gaussian.
__device__ __forceinline__ bool tile_reached(const TileEllipse& e, int tx, int ty) {
  if (e.S >= kNoBound) return true;
  if (e.S < 0.f) return false;
  const float x0 = (float)(tx * kTile) + 0.5f - e.px, y0 = (float)(ty * kTile) + 0.5f - e.py;
  return rect_min(e.A, e.B, e.C, e.kx, e.ky, x0, x0 + (float)(kTile - 1), y0, y0 + (float)(kTile - 1)) <= e.S;
}

__global__ void __launch_bounds__(kMarkThreads) mark_kernel(EmitArgs a, int smem_tiles) {
  extern __shared__ uint32_t s_tc[];
  pdl_wait();
  pdl_trigger();
  const int tid = threadIdx.x;
  for (int i = tid; i < smem_tiles; i += kMarkThreads) s_tc[i] = 0;
  __syncthreads();
  const uint32_t lane = lane_id(), warp = ((uint32_t)tid / 32) % (kPart / 32), half = (uint32_t)tid / kPart;
  const uint32_t* order = (a.order_sel && *a.order_sel) ? a.order_alt : a.order;
  const int pos = blockIdx.x * kPart + (int)(warp * 32 + lane);
  int4 r = make_int4(0, 0, 0, 0);
  uint32_t cnt = 0;
  // with a.cull: the ellipse {alpha >= 1/255} of this lane's Gaussian, for the tile test
  TileEllipse ell{0.f, 0.f, 0.f, -1.f, 0.f, 0.f, 0.f, 0.f};
  if (pos < a.n) {
    const uint32_t g = order ? order[pos] : (uint32_t)pos;
    r = a.rect[g];
    cnt = (uint32_t)max(0, r.z - r.x) * (uint32_t)max(0, r.w - r.y);
    if (cnt && (a.cull || (a.sorted_xy && half == 0))) {
      const float2 p = a.xy[g];
      const float4 co = a.conic_opacity[g];
      if (a.sorted_xy && half == 0) {  // the compositing reads the projected Gaussians by depth rank
        a.sorted_xy[pos] = p;
        a.sorted_co[pos] = co;
        a.sorted_rgb[3 * pos] = a.rgb[3 * g];
        a.sorted_rgb[3 * pos + 1] = a.rgb[3 * g + 1];
        a.sorted_rgb[3 * pos + 2] = a.rgb[3 * g + 2];
      }
      if (a.cull) ell = tile_ellipse(p, co);
    }
  }
  const uint32_t rw = (uint32_t)max(1, r.z - r.x);
  uint32_t incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= (uint32_t)d) incl += v;
  }
  const uint32_t excl = incl - cnt, total = __shfl_sync(0xffffffffu, incl, 31);
  uint32_t* col = a.bitmap + ((uint32_t)blockIdx.x * kPart + warp * 32) / 32;
  for (uint32_t j0 = 32 * half; j0 < total; j0 += 32 * kMarkHalves) {
    const uint32_t j = j0 + lane;
    // last lane whose offset is <= j (a lane with no tiles shares its offset with
    // the next lane, so it never wins)
    uint32_t lo = 0;
#pragma unroll
    for (uint32_t st = 16; st >= 1; st >>= 1) {
      const uint32_t e = __shfl_sync(0xffffffffu, excl, lo + st);
      if (e <= j) lo += st;
    }
    const int rx = __shfl_sync(0xffffffffu, r.x, lo), ry = __shfl_sync(0xffffffffu, r.y, lo);
    const uint32_t w = __shfl_sync(0xffffffffu, rw, lo), e0 = __shfl_sync(0xffffffffu, excl, lo);
    bool keep = j < total;
    uint32_t k = 0, row = 0;
    if (keep) {
      k = j - e0;
      row = rect_row(k, w);
    }
    if (a.cull) {  // uniform: the tile's pixel centres against the ellipse of the pair's Gaussian
      TileEllipse e;
      e.A = __shfl_sync(0xffffffffu, ell.A, lo); e.B = __shfl_sync(0xffffffffu, ell.B, lo);
      e.C = __shfl_sync(0xffffffffu, ell.C, lo); e.S = __shfl_sync(0xffffffffu, ell.S, lo);
      e.kx = __shfl_sync(0xffffffffu, ell.kx, lo); e.ky = __shfl_sync(0xffffffffu, ell.ky, lo);
      e.px = __shfl_sync(0xffffffffu, ell.px, lo); e.py = __shfl_sync(0xffffffffu, ell.py, lo);
      if (keep) keep = tile_reached(e, rx + (int)(k - row * w), ry + (int)row);
    }
    if (keep) {
      const uint32_t tile = (uint32_t)(ry + (int)row) * (uint32_t)a.tiles_x + (uint32_t)rx + (k - row * w);
      atomicOr(col + (size_t)tile * (size_t)a.words, 1u << lo);
      if (smem_tiles)
        atomicAdd(&s_tc[tile], 1u);
      else
        atomicAdd(&a.tile_count[tile], 1u);
    }
  }
  if (lane == 0 && half == 0 && total) atomicAdd(a.num_pairs, total);
  if (smem_tiles) {
    __syncthreads();
    for (int t = tid; t < smem_tiles; t += kMarkThreads) {
      const uint32_t v = s_tc[t];
      if (v) atomicAdd(&a.tile_count[t], v);
    }
  }
}

// One CTA per tile (longest lists first when a tile order is given).  Each step
// covers kXRounds * kXThreads uint4 of the row: in round i thread t holds uint4
// v0 + i * kXThreads + t, so every load is coalesced and the rank order is round
// by round, thread by thread.  The popcounts of rounds (0, 1) and (2, 3) are
// scanned as packed 16-bit pairs (at most 32768 bits per round), which gives every
// uint4 its list position with one barrier per step.  The thread stores the depth
// rank of each set bit there and zeroes the nonzero words; the walk ends at the
// row's last pair, so the row is all zero afterwards.  With ids the ranks are then
// replaced by the Gaussians (and keys) with unrolled gathers.  A tile whose range
// is (0, 0) because the pairs overflowed the buffers is only cleared.
constexpr int kXThreads = 256;
constexpr int kXRounds = 4;

__device__ __forceinline__ void extract_bits(const uint4& q, uint32_t r0, uint32_t o, uint32_t cnt,
                                             uint32_t* list) {
  const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint32_t m = wd[j];
    while (m) {  // the row holds exactly cnt bits; the bound only guards the range
      if (o < cnt) list[o] = r0 + 32u * (uint32_t)j + (uint32_t)(__ffs(m) - 1);
      ++o;
      m &= m - 1u;
    }
  }
}

__global__ void __launch_bounds__(kXThreads) extract_kernel(EmitArgs a, int ids) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t s_warp[2][2][kXThreads / 32];
  const int t = a.tile_order ? (int)a.tile_order[blockIdx.x] : (int)blockIdx.x;
  const uint32_t cnt = a.tile_count[t];
  if (cnt == 0) return;
  const uint2 rg = a.ranges[t];
  const bool write = rg.y > rg.x;
  uint32_t* list = a.values + rg.x;
  const int tid = threadIdx.x;
  const uint32_t lane = lane_id(), warp = (uint32_t)tid / 32;
  uint4* row = reinterpret_cast<uint4*>(a.bitmap + (size_t)t * (size_t)a.words);
  const int nvec = a.words >> 2;
  uint32_t done = 0;
  for (int v0 = 0, it = 0; v0 < nvec && done < cnt; v0 += kXRounds * kXThreads, ++it) {
    uint4 q[kXRounds];
    uint32_t c[kXRounds];
#pragma unroll
    for (int i = 0; i < kXRounds; ++i) {
      const int v = v0 + i * kXThreads + tid;
      q[i] = v < nvec ? row[v] : make_uint4(0u, 0u, 0u, 0u);
      c[i] = __popc(q[i].x) + __popc(q[i].y) + __popc(q[i].z) + __popc(q[i].w);
    }
    const uint32_t p01 = c[0] | (c[1] << 16), p23 = c[2] | (c[3] << 16);
    uint32_t i01 = p01, i23 = p23;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y01 = __shfl_up_sync(0xffffffffu, i01, d), y23 = __shfl_up_sync(0xffffffffu, i23, d);
      if (lane >= (uint32_t)d) {
        i01 += y01;
        i23 += y23;
      }
    }
    uint32_t(*sw)[kXThreads / 32] = s_warp[it & 1];  // two buffers: one barrier per step
    if (lane == 31) {
      sw[0][warp] = i01;
      sw[1][warp] = i23;
    }
    __syncthreads();
    uint32_t e01 = i01 - p01, e23 = i23 - p23, t01 = 0, t23 = 0;
#pragma unroll
    for (int w = 0; w < kXThreads / 32; ++w) {
      const uint32_t y01 = sw[0][w], y23 = sw[1][w];
      if ((uint32_t)w < warp) {
        e01 += y01;
        e23 += y23;
      }
      t01 += y01;
      t23 += y23;
    }
    const uint32_t tot[4] = {t01 & 0xffffu, t01 >> 16, t23 & 0xffffu, t23 >> 16};
    const uint32_t ex[4] = {e01 & 0xffffu, e01 >> 16, e23 & 0xffffu, e23 >> 16};
    uint32_t base = done;
#pragma unroll
    for (int i = 0; i < kXRounds; ++i) {
      if (c[i]) {
        const int v = v0 + i * kXThreads + tid;
        row[v] = make_uint4(0u, 0u, 0u, 0u);
        if (write) extract_bits(q[i], (uint32_t)v * 128u, base + ex[i], cnt, list);
      }
      base += tot[i];
    }
    done = base;
  }
  if (!write || !ids) return;
  __syncthreads();  // the ranks stored by the other threads are visible
  const uint32_t* order = (a.order_sel && *a.order_sel) ? a.order_alt : a.order;
  const uint32_t last = (uint32_t)a.n - 1u;  // ranks are < n: the clamp only guards the gathers
  constexpr int kU = 4;
  for (uint32_t i0 = (uint32_t)tid; i0 < cnt; i0 += kU * kXThreads) {
    uint32_t g[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const uint32_t i = i0 + (uint32_t)u * kXThreads;
      g[u] = i < cnt ? min(list[i], last) : 0u;
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) g[u] = order ? order[g[u]] : g[u];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const uint32_t i = i0 + (uint32_t)u * kXThreads;
      if (i < cnt) {
        list[i] = g[u];
        if (a.keys) a.keys[rg.x + i] = ((unsigned long long)t << 32) | __float_as_uint(a.depth[g[u]]);
      }
    }
  }
}

}  // namespace

int emit_parts(int n) { return (n + kPart - 1) / kPart; }

cudaError_t launch_scan_emit(const EmitArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  static PerDeviceFlag attr;
  cudaError_t e = once_per_device(attr, [] {
    return cudaFuncSetAttribute(scan_emit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * kEmitSmemTiles);
  });
  if (e != cudaSuccess) return e;
  const int st = a.n_tiles <= kEmitSmemTiles ? a.n_tiles : 0;
  return launch_pdl(scan_emit_kernel, emit_parts(a.n), kThreads, 4 * (size_t)st, s, a, st);
}

int bitmap_words(int n) { return ((n + 127) / 128) * 4; }

cudaError_t launch_mark_tiles(const EmitArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  static PerDeviceFlag attr;
  cudaError_t e = once_per_device(attr, [] {
    return cudaFuncSetAttribute(mark_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * kEmitSmemTiles);
  });
  if (e != cudaSuccess) return e;
  if (a.words < bitmap_words(a.n)) return cudaErrorInvalidValue;
  const int st = a.n_tiles <= kEmitSmemTiles ? a.n_tiles : 0;
  return launch_pdl(mark_kernel, emit_parts(a.n), kMarkThreads, 4 * (size_t)st, s, a, st);
}

cudaError_t launch_extract_tiles(const EmitArgs& a, bool ids, cudaStream_t s) {
  if (a.n <= 0 || a.n_tiles <= 0) return cudaSuccess;
  if (a.words < bitmap_words(a.n) || (a.words & 3)) return cudaErrorInvalidValue;
  return launch_pdl(extract_kernel, a.n_tiles, kXThreads, 0, s, a, ids ? 1 : 0);
}

cudaError_t launch_tile_scan(const uint32_t* tile_count, int n_tiles, uint32_t* num_pairs, uint2* ranges,
                             uint32_t* hist, int passes, uint32_t* order, cudaStream_t s, long long capacity,
                             uint32_t* status) {
  if (passes > kMaxPasses || n_tiles < 1) return cudaErrorInvalidValue;
  return launch_pdl(tile_scan_kernel, 1, kScanThreads, 0, s, tile_count, n_tiles, num_pairs, ranges, hist, passes, order,
                    capacity, status);
}

}  // namespace fs4d

namespace fs4d {
namespace {
__global__ void depth_keys_kernel(const float* __restrict__ depth, int n, unsigned long long* __restrict__ keys,
                                  uint32_t* __restrict__ vals) {
  pdl_wait();
  pdl_trigger();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = __float_as_uint(depth[i]);
  vals[i] = (uint32_t)i;
}
}  // namespace

cudaError_t launch_depth_keys(const float* depth, int n, unsigned long long* keys, uint32_t* vals, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  return launch_pdl(depth_keys_kernel, (n + 255) / 256, 256, 0, s, depth, n, keys, vals);
}

}  // namespace fs4d
