// Tile binning: one (tile | depth) key per (Gaussian, touched tile).
//
// A single pass does three jobs per 2048-Gaussian partition:
//   1. exclusive scan of the per-Gaussian tile counts, chained across CTAs by
//      decoupled look-back (the partition index comes from an atomic ticket, so
//      every predecessor a CTA waits on is already resident);
//   2. emission of the keys (tile_id << 32 | float bits of depth) and values
//      (Gaussian index) at the scanned offsets -- Gaussian order, then row-major
//      tile order, which is what makes the later stable sort break depth ties by
//      Gaussian index;
//   3. the 256-bin digit histograms of every radix pass, accumulated in shared
//      memory (depth digits once per Gaussian weighted by its count, tile digits
//      once per run of equal digits along a rect row) and merged with one global
//      atomic per non-empty bin.
// A second small kernel turns the sorted keys into per-tile [start, end) ranges.
#include "sync_util.cuh"

namespace fs4d {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kPart = kThreads * kItems;
constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;
constexpr int kMaxPasses = 8;

__global__ void __launch_bounds__(kThreads) scan_emit_kernel(EmitArgs a) {
  __shared__ uint32_t s_part;
  __shared__ uint32_t s_warp[kThreads / 32];
  __shared__ unsigned long long s_prefix;
  __shared__ uint32_t s_hist[kMaxPasses][256];
  const int tid = threadIdx.x;
  if (tid == 0) s_part = atomicAdd(a.part_counter, 1u);
  if (a.hist)
    for (int i = tid; i < kMaxPasses * 256; i += kThreads) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  const int part = (int)s_part;
  const int g0 = part * kPart + tid * kItems;

  uint32_t cnt[kItems];
  uint32_t sum = 0;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const int g = g0 + i;
    cnt[i] = 0;
    if (g < a.n) {
      const int4 r = a.rect[g];
      cnt[i] = (uint32_t)max(0, r.z - r.x) * (uint32_t)max(0, r.w - r.y);
    }
    sum += cnt[i];
  }
  // Block-wide exclusive scan of the per-thread sums.
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
  const uint32_t thread_excl = warp_excl + incl - sum;

  // Chain the partitions: publish this partition's total, then sum predecessors
  // until one with an inclusive prefix is found.
  if (tid == 0) {
    unsigned long long prefix = 0;
    if (part == 0) {
      st_relaxed_u64(&a.lookback[0], kFlagInc | block_total);
    } else {
      st_relaxed_u64(&a.lookback[part], kFlagAgg | block_total);
      int j = part - 1;
      uint32_t spins = 0;
      while (j >= 0) {
        const unsigned long long v = ld_relaxed_u64(&a.lookback[j]);
        const unsigned long long flag = v & ~kValMask;
        if (flag == 0) {
          if (++spins > kSpinLimit) {
            atomicOr(a.status, kStatusTimeout);
            break;
          }
          __nanosleep(32);
          continue;
        }
        prefix += v & kValMask;
        if (flag == kFlagInc) break;
        --j;
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

  unsigned long long off = s_prefix + thread_excl;
#pragma unroll 1
  for (int i = 0; i < kItems; ++i) {
    const int g = g0 + i;
    if (g >= a.n) break;
    a.offsets[g] = (uint32_t)off;
    const uint32_t c = cnt[i];
    if (c == 0) continue;
    const int4 r = a.rect[g];
    const uint32_t dbits = __float_as_uint(a.depth[g]);
    if (a.hist) {
      for (int p = 0; p < min(4, a.passes); ++p) atomicAdd(&s_hist[p][(dbits >> (8 * p)) & 255u], c);
    }
    const bool fits = (long long)(off + c) <= a.capacity;
    unsigned long long o = off;
    for (int ty = r.y; ty < r.w; ++ty) {
      const uint32_t row0 = (uint32_t)(ty * a.tiles_x);
      if (fits) {
        for (int tx = r.x; tx < r.z; ++tx) {
          const uint32_t tile = row0 + (uint32_t)tx;
          a.keys[o] = ((unsigned long long)tile << 32) | dbits;
          a.values[o] = (uint32_t)g;
          ++o;
        }
      }
      if (a.hist) {
        for (int p = 4; p < a.passes; ++p) {
          const int sh = 8 * (p - 4);
          uint32_t t = row0 + (uint32_t)r.x;
          const uint32_t t1 = row0 + (uint32_t)r.z - 1u;
          while (t <= t1) {
            const uint32_t run_end = min(t1, (((t >> sh) + 1u) << sh) - 1u);
            atomicAdd(&s_hist[p][(t >> sh) & 255u], run_end - t + 1u);
            t = run_end + 1u;
          }
        }
      }
    }
    off += c;
  }
  if (a.hist) {
    __syncthreads();
    for (int i = tid; i < a.passes * 256; i += kThreads) {
      const uint32_t v = (&s_hist[0][0])[i];
      if (v) atomicAdd(&a.hist[i], v);
    }
  }
}

__global__ void __launch_bounds__(256) ranges_kernel(const unsigned long long* __restrict__ keys,
                                                     const uint32_t* __restrict__ n_dev, long long n_bound,
                                                     uint2* __restrict__ ranges, uint32_t n_tiles) {
  const long long n = n_dev ? (long long)*n_dev : n_bound;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || i >= n_bound) return;
  const uint32_t tile = (uint32_t)(keys[i] >> 32);
  if (tile >= n_tiles) return;
  if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != tile) ranges[tile].x = (uint32_t)i;
  if (i == n - 1 || (uint32_t)(keys[i + 1] >> 32) != tile) ranges[tile].y = (uint32_t)(i + 1);
}

}  // namespace

int emit_parts(int n) { return (n + kPart - 1) / kPart; }

cudaError_t launch_scan_emit(const EmitArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (a.passes > kMaxPasses) return cudaErrorInvalidValue;
  scan_emit_kernel<<<emit_parts(a.n), kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_ranges(const unsigned long long* keys, const uint32_t* n_dev, long long n_bound, uint2* ranges,
                          int n_tiles, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)n_tiles, s);
  if (e != cudaSuccess || n_bound <= 0) return e;
  ranges_kernel<<<(unsigned)((n_bound + 255) / 256), 256, 0, s>>>(keys, n_dev, n_bound, ranges, (uint32_t)n_tiles);
  return cudaGetLastError();
}

}  // namespace fs4d
