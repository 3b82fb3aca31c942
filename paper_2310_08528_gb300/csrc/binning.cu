// Tile binning: one (tile | depth) key per (Gaussian, touched tile).
//
// Gaussians are visited in a given order (the depth-sorted order, so that a
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
          if (++spins > kSpinLimit) {
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
      key = ((unsigned long long)tile << 32) | s_dbits[lo];
      const unsigned long long out = prefix + j;
      if ((long long)out < a.capacity) {
        a.keys[out] = key;
        a.values[out] = s_gid[lo];
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
                                                                 const uint32_t* __restrict__ num_pairs,
                                                                 uint2* __restrict__ ranges, uint32_t* __restrict__ hist,
                                                                 int passes, uint32_t* __restrict__ order) {
  __shared__ uint32_t s_warp[kScanThreads / 32];
  __shared__ uint32_t s_hist[kMaxPasses][256];
  __shared__ uint32_t s_len[33];          // tiles per length class floor(log2(count)) + 1 (0: empty)
  const int tid = threadIdx.x;
  const uint32_t lane = lane_id(), warp = tid / 32;
  for (int i = tid; i < kMaxPasses * 256; i += kScanThreads) (&s_hist[0][0])[i] = 0;
  if (tid < 33) s_len[tid] = 0;
  const bool overflow = num_pairs[1] == 0u && num_pairs[0] != 0u;
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
  for (int w = 0; w < (int)warp; ++w) run += s_warp[w];
  for (int t = t0; t < t1; ++t) {
    const uint32_t c = tile_count[t];
    ranges[t] = (overflow || c == 0) ? make_uint2(0u, 0u) : make_uint2(run, run + c);
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
    // the longest lists start first and do not form the tail.
    for (int t = t0; t < t1; ++t) {
      const uint32_t c = overflow ? 0u : tile_count[t];
      atomicAdd(&s_len[32 - (c ? 32 - __clz(c) : 0)], 1u);
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
    for (int t = t0; t < t1; ++t) {
      const uint32_t c = overflow ? 0u : tile_count[t];
      order[atomicAdd(&s_len[32 - (c ? 32 - __clz(c) : 0)], 1u)] = (uint32_t)t;
    }
  }
}

}  // namespace

int emit_parts(int n) { return (n + kPart - 1) / kPart; }

cudaError_t launch_scan_emit(const EmitArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(scan_emit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * kEmitSmemTiles);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int st = a.n_tiles <= kEmitSmemTiles ? a.n_tiles : 0;
  scan_emit_kernel<<<emit_parts(a.n), kThreads, 4 * (size_t)st, s>>>(a, st);
  return cudaGetLastError();
}

cudaError_t launch_tile_scan(const uint32_t* tile_count, int n_tiles, const uint32_t* num_pairs, uint2* ranges,
                             uint32_t* hist, int passes, uint32_t* order, cudaStream_t s) {
  if (passes > kMaxPasses || n_tiles < 1) return cudaErrorInvalidValue;
  tile_scan_kernel<<<1, kScanThreads, 0, s>>>(tile_count, n_tiles, num_pairs, ranges, hist, passes, order);
  return cudaGetLastError();
}

}  // namespace fs4d

namespace fs4d {
namespace {
__global__ void depth_keys_kernel(const float* __restrict__ depth, int n, unsigned long long* __restrict__ keys,
                                  uint32_t* __restrict__ vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = __float_as_uint(depth[i]);
  vals[i] = (uint32_t)i;
}
}  // namespace

cudaError_t launch_depth_keys(const float* depth, int n, unsigned long long* keys, uint32_t* vals, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  depth_keys_kernel<<<(n + 255) / 256, 256, 0, s>>>(depth, n, keys, vals);
  return cudaGetLastError();
}

}  // namespace fs4d
