// Stable LSD radix sort of (64-bit key, 32-bit value) pairs, one-sweep style:
//  - one histogram pass produces the 256-bin digit counts of EVERY radix pass at
//    once (skipped when the binning kernel already produced them);
//  - then one kernel per 8-bit digit.  Each CTA takes a 4096-pair partition by
//    atomic ticket, ranks its keys stably (warp-striped order, ballot-multisplit
//    peers per digit, warp offsets chained through shared memory), publishes its
//    per-digit counts and resolves its global per-digit offsets by decoupled
//    look-back on its predecessors, then scatters through shared memory so that
//    runs of equal digits are written contiguously;
//  - or, for a sort whose 1024-key partitions are all resident at once (a frame's
//    depth sort of up to ~150k keys), every pass in one launch: CTA b owns
//    partition b in every pass and a bounded grid barrier separates the passes.
// Only the key bits that can differ are sorted.  A frame sorts the N float32
// depths (32 bits in 4 passes; a pass whose digit is the same for every key moves
// nothing) and, on the key-emission route, the pairs on their tile bits only (the
// pairs are emitted in depth order, so 2500 tiles sort 12 bits in 2 passes).
#include <algorithm>

#include "sync_util.cuh"

namespace fs4d {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItemsLarge = 16;  // keys per thread for large sorts (4096 per partition)
constexpr int kItemsSmall = 4;   // ... and for sorts of a few 100k keys (1024 per partition)
constexpr int kPartPairs = kThreads * kItemsLarge;
constexpr int kPartPairsSmall = kThreads * kItemsSmall;
constexpr int kRadix = 256;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kValMask = (1u << 30) - 1u;
constexpr int kMaxPasses = 8;

__global__ void __launch_bounds__(256) hist_kernel(const unsigned long long* __restrict__ keys,
                                                   const uint32_t* __restrict__ n_dev, long long n_bound,
                                                   int first_bit, int key_bits, int passes,
                                                   uint32_t* __restrict__ hist) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t s_hist[kMaxPasses][kRadix];
  for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += blockDim.x) (&s_hist[0][0])[i] = 0;
  __syncthreads();
  const long long n = n_dev ? min((long long)*n_dev, n_bound) : n_bound;
  const uint32_t lane_lt = lanemask_lt();
  for (long long base = (long long)blockIdx.x * blockDim.x; base < n; base += (long long)gridDim.x * blockDim.x) {
    const long long i = base + threadIdx.x;
    const bool valid = i < n;
    const unsigned long long k = valid ? keys[i] : 0ull;
    for (int p = 0; p < passes; ++p) {
      const int bits = min(8, key_bits - 8 * p);
      const uint32_t d = valid ? (uint32_t)(k >> (first_bit + 8 * p)) & ((1u << bits) - 1u) : 256u;
      const uint32_t peers = digit_peers(d, d < 256u, bits);
      if (d < 256u && (peers & lane_lt) == 0) atomicAdd(&s_hist[p][d], (uint32_t)__popc(peers));
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
    const uint32_t v = (&s_hist[0][0])[i];
    if (v) atomicAdd(&hist[i], v);
  }
}

struct PassArgs {
  const unsigned long long* keys_in;   // with sel_in: buffer A, the other one is B
  const uint32_t* values_in;
  unsigned long long* keys_out;
  uint32_t* values_out;
  const uint32_t* sel_in;   // optional: 1 if this pass's input is in B (the *_out pointers)
  uint32_t* sel_out;        //   where the pass records where its output is
  const uint32_t* n_dev;
  long long n_bound;
  int shift;
  const uint32_t* hist;     // this pass's 256 counts
  uint32_t* lookback;       // this pass's [parts][256], zeroed
  uint32_t* part_counter;   // this pass's ticket, zeroed
  uint32_t* status;
  uint32_t spin_limit;      // polls of the look-back wait before it gives up
  int bits;                 // significant bits of this pass's digit (<= 8; the key's last bits)
};

template <int ITEMS>
struct PassSmem {
  unsigned long long keys[kThreads * ITEMS];
  uint32_t values[kThreads * ITEMS];
  uint32_t warp_cnt[kWarps][kRadix];
  uint32_t global_off[kRadix];   // exclusive scan of the global histogram
  uint32_t block_off[kRadix];    // exclusive scan of this partition's counts
  uint32_t prev_off[kRadix];     // sum of predecessors' counts (look-back)
  uint32_t scan_tmp[kWarps];
  uint32_t part;
};

// Exclusive scan of one value per thread across the 256-thread block.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* tmp) {
  const uint32_t lane = lane_id(), warp = threadIdx.x / 32;
  uint32_t incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= (uint32_t)d) incl += t;
  }
  if (lane == 31) tmp[warp] = incl;
  __syncthreads();
  uint32_t base = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w)
    if ((uint32_t)w < warp) base += tmp[w];
  __syncthreads();
  return base + incl - v;
}

// One pass over partition `part` (elements [base, base + kThreads * ITEMS) of n):
// rank the keys stably within the CTA, publish the digit counts, sort locally,
// resolve the global offsets by decoupled look-back and scatter.  h = the
// pass's global count of digit tid.  Every thread of the CTA calls it.
template <int ITEMS, bool VALS>
__device__ __forceinline__ void onesweep_pass(PassSmem<ITEMS>& sm, const PassArgs& a, uint32_t part, long long base,
                                              long long n, uint32_t h, const unsigned long long* keys_in,
                                              const uint32_t* values_in, unsigned long long* keys_out,
                                              uint32_t* values_out) {
  constexpr int kItems = ITEMS;
  constexpr int kPartPairs = kThreads * ITEMS;
  const int tid = threadIdx.x;
  const uint32_t lane = lane_id(), warp = tid / 32;
  // Global offset of each digit.
  sm.global_off[tid] = block_excl_scan(h, sm.scan_tmp);

  // Load (warp-striped: item i of lane l is element base + warp*512 + i*32 + l)
  // and rank within the warp.
  unsigned long long k[kItems];
  uint32_t v[kItems], rank[kItems];
  uint16_t dig[kItems];
  const uint32_t lt = lanemask_lt();
  // all loads first, so that every thread has its kItems requests in flight at once
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const long long idx = base + (long long)warp * (kItems * 32) + i * 32 + lane;
    const bool valid = idx < n;
    k[i] = valid ? keys_in[idx] : 0ull;
    v[i] = (VALS && valid) ? values_in[idx] : 0u;
    dig[i] = (uint16_t)(valid ? (uint32_t)(k[i] >> a.shift) & ((1u << a.bits) - 1u) : 256u);
  }
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const uint32_t d = dig[i];
    const uint32_t peers = digit_peers(d, d < 256u, a.bits);
    uint32_t before = 0;
    if (d < 256u) before = sm.warp_cnt[warp][d];
    __syncwarp();
    rank[i] = before + (uint32_t)__popc(peers & lt);
    if (d < 256u && (peers & lt) == 0) sm.warp_cnt[warp][d] = before + (uint32_t)__popc(peers);
    __syncwarp();
  }
  __syncthreads();

  // Per digit (thread tid = digit): chain the warps, publish this partition's
  // count, then sort locally through shared memory before looking back, so the
  // look-back runs with the keys already out of registers.
  uint32_t total = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const uint32_t c = sm.warp_cnt[w][tid];
    sm.warp_cnt[w][tid] = total;
    total += c;
  }
  uint32_t* lb = a.lookback + (size_t)part * kRadix + tid;
  st_relaxed_u32(lb, (part == 0 ? kFlagInc : kFlagAgg) | total);
  sm.block_off[tid] = block_excl_scan(total, sm.scan_tmp);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const uint32_t d = dig[i];
    if (d < 256u) {
      const uint32_t pos = sm.block_off[d] + sm.warp_cnt[warp][d] + rank[i];
      sm.keys[pos] = k[i];
      if (VALS) sm.values[pos] = v[i];
    }
  }

  // Look-back: read up to 32 predecessors at once (independent loads), then
  // consume them nearest first until an inclusive prefix is found.  All
  // partitions publish at about the same time, so a wide window keeps the
  // number of dependent rounds small.
  uint32_t prev = 0;
  if (part > 0) {
    constexpr int kWin = 32;
    long long j = (long long)part - 1;
    uint32_t spins = 0;
    bool found = false;
    while (j >= 0 && !found) {
      const int cnt = (int)min((long long)kWin, j + 1);
      uint32_t wv[kWin];
#pragma unroll
      for (int i = 0; i < kWin; ++i)
        if (i < cnt) wv[i] = ld_relaxed_u32(a.lookback + (size_t)(j - i) * kRadix + tid);
      int used = 0;
#pragma unroll
      for (int i = 0; i < kWin; ++i) {
        if (i >= cnt || found) break;
        const uint32_t flag = wv[i] & ~kValMask;
        if (flag == 0) break;  // not published yet: poll again from here
        prev += wv[i] & kValMask;
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
    st_relaxed_u32(lb, kFlagInc | ((prev + total) & kValMask));
  }
  sm.prev_off[tid] = sm.global_off[tid] + prev - sm.block_off[tid];
  __syncthreads();

  // Scatter: consecutive slots of one digit go to consecutive addresses
  // (prev_off holds global + look-back - local offset of each digit).
  const int m = (int)min((long long)kPartPairs, n - base);
  for (int j = tid; j < m; j += kThreads) {
    const unsigned long long key = sm.keys[j];
    const uint32_t d = (uint32_t)(key >> a.shift) & ((1u << a.bits) - 1u);
    const uint32_t out = sm.prev_off[d] + (uint32_t)j;
    if ((long long)out < n) {  // always true when the histogram matches the keys
      keys_out[out] = key;
      if (VALS) values_out[out] = sm.values[j];
    }
  }
}


// VALS = false: keys only (values_* unused); the key carries its payload.
template <int ITEMS, bool VALS>
__global__ void __launch_bounds__(kThreads) onesweep_kernel(PassArgs a) {
  constexpr int kPartPairs = kThreads * ITEMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PassSmem<ITEMS>& sm = *reinterpret_cast<PassSmem<ITEMS>*>(smem_raw);
  const int tid = threadIdx.x;
  pdl_wait();
  pdl_trigger();
  if (tid == 0) sm.part = atomicAdd(a.part_counter, 1u);
  // independent of the ticket: issued while it is in flight
  const long long n = a.n_dev ? min((long long)*a.n_dev, a.n_bound) : a.n_bound;
  const uint32_t h = a.hist[tid];
  const bool in_b = a.sel_in && *a.sel_in;
  const unsigned long long* keys_in = in_b ? a.keys_out : a.keys_in;
  const uint32_t* values_in = in_b ? a.values_out : a.values_in;
  unsigned long long* keys_out = in_b ? const_cast<unsigned long long*>(a.keys_in) : a.keys_out;
  uint32_t* values_out = in_b ? const_cast<uint32_t*>(a.values_in) : a.values_out;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) sm.warp_cnt[w][tid] = 0;
  __syncthreads();
  const uint32_t part = sm.part;
  const long long base = (long long)part * kPartPairs;
  if (base >= n) return;  // uniform across the CTA
  // A pass whose digit is the same for every key keeps the order: with a
  // selection word it only records that the data stayed put, else it copies.
  const bool trivial = __syncthreads_or((long long)h == n);
  if (a.sel_out && part == 0 && tid == 0) *a.sel_out = (uint32_t)in_b ^ (trivial ? 0u : 1u);
  if (trivial) {
    if (a.sel_out) return;
    const long long m = min((long long)kPartPairs, n - base);
    for (long long i = tid; i < m; i += kThreads) {
      keys_out[base + i] = keys_in[base + i];
      if (VALS) values_out[base + i] = values_in[base + i];
    }
    return;
  }

  onesweep_pass<ITEMS, VALS>(sm, a, part, base, n, h, keys_in, values_in, keys_out, values_out);
}

// Grid-wide barrier of a kernel whose CTAs are all resident: arrival counter
// (zero before the launch), bounded spin by thread 0 (on giving up it records
// kStatusTimeout and lets the CTA go on).
__device__ __forceinline__ void grid_sync(uint32_t* counter, uint32_t target, uint32_t* status, uint32_t spin_limit) {
  __syncthreads();  // the CTA's stores of this pass are issued
  if (threadIdx.x == 0) {
    __threadfence();  // ... and visible device-wide before the arrival
    atomicAdd(counter, 1u);
    uint32_t spins = 0;
    while (ld_relaxed_u32(counter) < target) {
      if (++spins > spin_limit) {
        atomicOr(status, kStatusTimeout);
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
}

// Every pass of a sort small enough that all its 1024-key partitions are resident
// at once (a frame's depth sort: 100k keys, 98 partitions) in one launch: CTA b owns
// partition b in every pass and a grid barrier separates the passes, so the passes
// need no further launch and no ticket.  A pass whose digit every key shares moves
// nothing (the same decision in every CTA: it comes from the global histogram);
// *a.sel_out records whether the result ended in the alternate buffers.
__global__ void __launch_bounds__(kThreads) onesweep_fused_kernel(PassArgs a, int passes, int first_bit,
                                                                  int key_bits, uint32_t* grid_counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PassSmem<kItemsSmall>& sm = *reinterpret_cast<PassSmem<kItemsSmall>*>(smem_raw);
  const int tid = threadIdx.x;
  pdl_wait();
  pdl_trigger();  // (fires once every CTA of this grid runs: they are all resident)
  const long long n = a.n_bound;
  const uint32_t part = blockIdx.x;
  const long long base = (long long)part * kPartPairsSmall;
  uint32_t cur = 0, barriers = 0;
  for (int p = 0; p < passes; ++p) {
    const uint32_t h = a.hist[p * kRadix + tid];
#pragma unroll
    for (int w = 0; w < kWarps; ++w) sm.warp_cnt[w][tid] = 0;
    if (__syncthreads_or((long long)h == n)) continue;  // trivial pass (uniform)
    if (barriers > 0) grid_sync(grid_counter, barriers * gridDim.x, a.status, a.spin_limit);  // the last pass is out
    PassArgs pa = a;
    pa.shift = first_bit + 8 * p;
    pa.bits = min(8, key_bits - 8 * p);
    pa.lookback = a.lookback + (size_t)p * gridDim.x * kRadix;
    const unsigned long long* kin = cur ? a.keys_out : a.keys_in;
    const uint32_t* vin = cur ? a.values_out : a.values_in;
    unsigned long long* kout = cur ? const_cast<unsigned long long*>(a.keys_in) : a.keys_out;
    uint32_t* vout = cur ? const_cast<uint32_t*>(a.values_in) : a.values_out;
    onesweep_pass<kItemsSmall, true>(sm, pa, part, base, n, h, kin, vin, kout, vout);
    cur ^= 1u;
    ++barriers;
  }
  if (part == 0 && tid == 0) *a.sel_out = cur;
}

// ---------------------------------------------------------------- large sorts
// The same pass as a persistent kernel for large sorts: one CTA per resident slot
// loops over 4096-key partitions in ticket order and, while it ranks, looks back
// and scatters partition p, the keys (and values) of its next partition are already
// on their way into the other half of a double buffer in shared memory (cp.async),
// so the DRAM latency of the loads overlaps the work of the previous partition.
// The next ticket is taken before the current partition is finished; every ticket
// below it belongs to a CTA that is running or done, and a CTA works through its
// tickets in increasing order, so the lowest unfinished partition is always being
// worked on and every look-back wait ends.
constexpr int kPItems = 16;
constexpr int kPPart = kThreads * kPItems;  // 4096

template <bool VALS>
struct PersistSmem {
  unsigned long long keys[2][kPPart];  // loaded keys; the current half is reused for the local sort
  uint32_t values[VALS ? 2 : 1][VALS ? kPPart : 1];
  uint32_t warp_cnt[kWarps][kRadix];
  uint32_t global_off[kRadix];
  uint32_t block_off[kRadix];
  uint32_t prev_off[kRadix];
  uint32_t scan_tmp[kWarps];
  uint32_t part[2];
};

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, uint32_t src_bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(src_bytes) : "memory");
}

// Queue the loads of partition `part` (elements [base, base + m)) into half `b`:
// 16-byte chunks, the ragged end zero-filled (its source address clamped to the
// partition's first element, which is valid).
template <bool VALS>
__device__ __forceinline__ void persist_load(PersistSmem<VALS>& sm, int b, const unsigned long long* keys_in,
                                             const uint32_t* values_in, long long base, int m) {
  const int tid = threadIdx.x;
  for (int c = tid; c < kPPart / 2; c += kThreads) {  // 2 keys per chunk
    const int e = 2 * c;
    const int valid = max(0, min(2, m - e));
    const unsigned long long* src = keys_in + base + (valid ? e : 0);
    cp_async16(&sm.keys[b][e], src, 8u * (uint32_t)valid);
  }
  if (VALS) {
    for (int c = tid; c < kPPart / 4; c += kThreads) {  // 4 values per chunk
      const int e = 4 * c;
      const int valid = max(0, min(4, m - e));
      const uint32_t* src = values_in + base + (valid ? e : 0);
      cp_async16(&sm.values[b][e], src, 4u * (uint32_t)valid);
    }
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <bool VALS>
__global__ void __launch_bounds__(kThreads, 2) onesweep_persist_kernel(PassArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PersistSmem<VALS>& sm = *reinterpret_cast<PersistSmem<VALS>*>(smem_raw);
  const int tid = threadIdx.x;
  const uint32_t lane = lane_id(), warp = tid / 32;
  pdl_wait();
  pdl_trigger();
  const long long n = a.n_dev ? min((long long)*a.n_dev, a.n_bound) : a.n_bound;
  const long long parts = (n + kPPart - 1) / kPPart;
  if (tid == 0) sm.part[0] = atomicAdd(a.part_counter, 1u);
  const uint32_t h = a.hist[tid];
  sm.global_off[tid] = block_excl_scan(h, sm.scan_tmp);  // (its barriers publish sm.part[0])
  long long cur = sm.part[0];
  if (cur >= parts) return;  // uniform
  if (__syncthreads_or((long long)h == n)) {
    // every key has the same digit: the pass keeps the order (copy this CTA's partitions)
    for (; cur < parts;) {
      const long long base = cur * kPPart;
      const long long m = min((long long)kPPart, n - base);
      for (long long i = tid; i < m; i += kThreads) {
        a.keys_out[base + i] = a.keys_in[base + i];
        if (VALS) a.values_out[base + i] = a.values_in[base + i];
      }
      __syncthreads();
      if (tid == 0) sm.part[0] = atomicAdd(a.part_counter, 1u);
      __syncthreads();
      cur = sm.part[0];
    }
    return;
  }
  persist_load<VALS>(sm, 0, a.keys_in, a.values_in, cur * kPPart, (int)min((long long)kPPart, n - cur * kPPart));
  const uint32_t lt = lanemask_lt();
  for (int it = 0;; ++it) {
    const int b = it & 1;
    // the next partition's ticket, and its loads into the other half
    if (tid == 0) sm.part[b ^ 1] = atomicAdd(a.part_counter, 1u);
#pragma unroll
    for (int w = 0; w < kWarps; ++w) sm.warp_cnt[w][tid] = 0;
    __syncthreads();  // the other half was last read by the previous partition's scatter
    const long long next = sm.part[b ^ 1];
    if (next < parts) {
      persist_load<VALS>(sm, b ^ 1, a.keys_in, a.values_in, next * kPPart,
                         (int)min((long long)kPPart, n - next * kPPart));
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();  // this partition's keys are in half b
    const long long base = cur * kPPart;
    const int m = (int)min((long long)kPPart, n - base);
    // rank within the warp (warp-striped: item i of lane l is element warp*512 + i*32 + l)
    unsigned long long k[kPItems];
    uint32_t v[kPItems], rank[kPItems];
    uint16_t dig[kPItems];
#pragma unroll
    for (int i = 0; i < kPItems; ++i) {
      const int e = (int)warp * (kPItems * 32) + i * 32 + (int)lane;
      const bool valid = e < m;
      k[i] = sm.keys[b][e];
      v[i] = VALS ? sm.values[b][e] : 0u;
      dig[i] = (uint16_t)(valid ? (uint32_t)(k[i] >> a.shift) & ((1u << a.bits) - 1u) : 256u);
    }
#pragma unroll
    for (int i = 0; i < kPItems; ++i) {
      const uint32_t d = dig[i];
      const uint32_t peers = digit_peers(d, d < 256u, a.bits);
      uint32_t before = 0;
      if (d < 256u) before = sm.warp_cnt[warp][d];
      __syncwarp();
      rank[i] = before + (uint32_t)__popc(peers & lt);
      if (d < 256u && (peers & lt) == 0) sm.warp_cnt[warp][d] = before + (uint32_t)__popc(peers);
      __syncwarp();
    }
    __syncthreads();  // every key of half b is in registers: the half is free for the local sort
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
      const uint32_t c = sm.warp_cnt[w][tid];
      sm.warp_cnt[w][tid] = total;
      total += c;
    }
    uint32_t* lb = a.lookback + (size_t)cur * kRadix + tid;
    st_relaxed_u32(lb, (cur == 0 ? kFlagInc : kFlagAgg) | total);
    sm.block_off[tid] = block_excl_scan(total, sm.scan_tmp);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kPItems; ++i) {
      const uint32_t d = dig[i];
      if (d < 256u) {
        const uint32_t pos = sm.block_off[d] + sm.warp_cnt[warp][d] + rank[i];
        sm.keys[b][pos] = k[i];
        if (VALS) sm.values[b][pos] = v[i];
      }
    }
    // look-back (one thread per digit, 32 predecessors per round of independent loads)
    uint32_t prev = 0;
    if (cur > 0) {
      constexpr int kWin = 32;
      long long j = cur - 1;
      uint32_t spins = 0;
      bool found = false;
      while (j >= 0 && !found) {
        const int cnt = (int)min((long long)kWin, j + 1);
        uint32_t wv[kWin];
#pragma unroll
        for (int i = 0; i < kWin; ++i)
          if (i < cnt) wv[i] = ld_relaxed_u32(a.lookback + (size_t)(j - i) * kRadix + tid);
        int used = 0;
#pragma unroll
        for (int i = 0; i < kWin; ++i) {
          if (i >= cnt || found) break;
          const uint32_t flag = wv[i] & ~kValMask;
          if (flag == 0) break;
          prev += wv[i] & kValMask;
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
      st_relaxed_u32(lb, kFlagInc | ((prev + total) & kValMask));
    }
    sm.prev_off[tid] = sm.global_off[tid] + prev - sm.block_off[tid];  // global + look-back - local
    __syncthreads();
    for (int j2 = tid; j2 < m; j2 += kThreads) {
      const unsigned long long key = sm.keys[b][j2];
      const uint32_t d = (uint32_t)(key >> a.shift) & ((1u << a.bits) - 1u);
      const uint32_t out = sm.prev_off[d] + (uint32_t)j2;
      if ((long long)out < n) {  // always true when the histogram matches the keys
        a.keys_out[out] = key;
        if (VALS) a.values_out[out] = sm.values[b][j2];
      }
    }
    cur = next;
    if (cur >= parts) break;
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

}  // namespace

int sort_passes(int key_bits) { return (key_bits + 7) / 8; }

int device_sm_count() {
  static std::atomic<int> sms[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
  int v = sms[dev].load(std::memory_order_relaxed);
  if (v <= 0) {
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (v <= 0) v = 1;
    sms[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}
// Partitions a sort of n keys may use: small partitions up to 2^19 keys, large
// ones above (the look-back tables are sized by this).
long long sort_parts(long long n) {
  const long long small = (std::min(n, 1ll << 19) + kPartPairsSmall - 1) / kPartPairsSmall;
  return std::max(small, (n + kPartPairs - 1) / kPartPairs);
}

cudaError_t launch_sort(unsigned long long* keys, uint32_t* values, unsigned long long* keys_alt,
                        uint32_t* values_alt, const uint32_t* n_dev, long long n_bound, int first_bit,
                        int key_bits, bool hist_ready, const SortWork& work, uint32_t* status, cudaStream_t s,
                        bool* result_in_alt, const uint32_t** result_sel) {
  *result_in_alt = false;
  if (result_sel) *result_sel = nullptr;
  const int passes = sort_passes(key_bits);
  if (n_bound <= 0 || passes == 0) return cudaSuccess;
  if (passes > kMaxPasses) return cudaErrorInvalidValue;
  // small partitions keep enough CTAs in flight for a few 100k keys; large ones
  // amortise the look-back for millions (and fit a fixed look-back table)
  const long long parts_small = (n_bound + kPartPairsSmall - 1) / kPartPairsSmall;
  const bool small = n_bound <= (1ll << 19) && parts_small <= work.max_parts;
  const long long parts = small ? parts_small : (n_bound + kPartPairs - 1) / kPartPairs;
  if (parts > work.max_parts || n_bound > (long long)kValMask) return cudaErrorInvalidValue;
  static PerDeviceFlag attr;
  cudaError_t e = once_per_device(attr, [] {
    const int large = (int)sizeof(PassSmem<kItemsLarge>), small_b = (int)sizeof(PassSmem<kItemsSmall>);
    cudaError_t r = cudaFuncSetAttribute(onesweep_kernel<kItemsLarge, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, large);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(onesweep_kernel<kItemsSmall, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               small_b);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(onesweep_kernel<kItemsLarge, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               large);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(onesweep_kernel<kItemsSmall, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               small_b);
    return r;
  });
  if (e != cudaSuccess) return e;
  if (!work.prezeroed) {
    // tickets [0, kMaxPasses) and selection words [kMaxPasses, 2 kMaxPasses + 1)
    e = cudaMemsetAsync(work.part_counters, 0, sizeof(uint32_t) * (2 * kMaxPasses + 1), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(work.lookback, 0, sizeof(uint32_t) * (size_t)passes * parts * kRadix, s);
    if (e != cudaSuccess) return e;
  }
  if (!hist_ready) {
    e = cudaMemsetAsync(work.hist, 0, sizeof(uint32_t) * kMaxPasses * kRadix, s);
    if (e != cudaSuccess) return e;
    const int blocks = (int)min((n_bound + 1023) / 1024, (long long)device_sm_count() * 8);
    e = launch_pdl(hist_kernel, blocks, 256, 0, s, keys, n_dev, n_bound, first_bit, key_bits, passes, work.hist);
    if (e != cudaSuccess) return e;
  }
  unsigned long long* kin = keys;
  uint32_t* vin = values;
  unsigned long long* kout = keys_alt;
  uint32_t* vout = values_alt;
  uint32_t* sel = result_sel ? work.part_counters + kMaxPasses : nullptr;
  // every pass in one launch when all the partitions fit on the GPU at once
  if (small && !n_dev && sel && values && work.prezeroed && work.grid_counter) {
    static std::atomic<int> per_sm[kMaxDevices] = {};
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    int fit = per_sm[dev].load(std::memory_order_relaxed);
    if (fit <= 0) {
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, onesweep_fused_kernel, kThreads,
                                                         sizeof(PassSmem<kItemsSmall>));
      if (e != cudaSuccess) return e;
      per_sm[dev].store(std::max(fit, 1), std::memory_order_relaxed);
    }
    // (half of what fits, so that a kernel still running beside it cannot keep a partition out)
    if (parts * 2 <= (long long)fit * device_sm_count()) {
      PassArgs pa{};
      pa.keys_in = keys; pa.values_in = values; pa.keys_out = keys_alt; pa.values_out = values_alt;
      pa.sel_out = sel;
      pa.n_bound = n_bound;
      pa.hist = work.hist;
      pa.lookback = work.lookback;
      pa.status = status;
      pa.spin_limit = work.spin_limit;
      e = launch_pdl(onesweep_fused_kernel, (unsigned)parts, kThreads, sizeof(PassSmem<kItemsSmall>), s, pa, passes,
                     first_bit, key_bits, work.grid_counter);
      if (e != cudaSuccess) return e;
      *result_sel = sel;
      return cudaSuccess;
    }
  }
  // large sorts without device-side buffer selection: the persistent, prefetching pass
  const bool persist = !small && !sel;
  int persist_grid = 0;
  if (persist) {
    const bool vals = values != nullptr;
    const size_t smem = vals ? sizeof(PersistSmem<true>) : sizeof(PersistSmem<false>);
    static PerDeviceFlag pattr;
    e = once_per_device(pattr, [] {
      cudaError_t r = cudaFuncSetAttribute(onesweep_persist_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sizeof(PersistSmem<true>));
      if (r == cudaSuccess)
        r = cudaFuncSetAttribute(onesweep_persist_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(PersistSmem<false>));
      return r;
    });
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = vals ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, onesweep_persist_kernel<true>, kThreads, smem)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, onesweep_persist_kernel<false>, kThreads, smem);
    if (e != cudaSuccess) return e;
    persist_grid = (int)std::min<long long>(parts, (long long)std::max(per_sm, 1) * device_sm_count());
  }
  for (int p = 0; p < passes; ++p) {
    PassArgs pa;
    if (sel) {  // buffers fixed as A = (keys, values), B = alt; the device tracks where the data is
      pa.keys_in = keys; pa.values_in = values; pa.keys_out = keys_alt; pa.values_out = values_alt;
      pa.sel_in = sel + p;
      pa.sel_out = sel + p + 1;
    } else {
      pa.keys_in = kin; pa.values_in = vin; pa.keys_out = kout; pa.values_out = vout;
      pa.sel_in = nullptr;
      pa.sel_out = nullptr;
    }
    pa.n_dev = n_dev; pa.n_bound = n_bound; pa.shift = first_bit + 8 * p;
    pa.bits = std::min(8, key_bits - 8 * p);
    pa.hist = work.hist + p * kRadix;
    pa.lookback = work.lookback + (size_t)p * parts * kRadix;
    pa.part_counter = work.part_counters + p;
    pa.status = status;
    pa.spin_limit = work.spin_limit;
    const bool vals = values != nullptr;
    if (persist)
      e = vals ? launch_pdl(onesweep_persist_kernel<true>, (unsigned)persist_grid, kThreads,
                            sizeof(PersistSmem<true>), s, pa)
               : launch_pdl(onesweep_persist_kernel<false>, (unsigned)persist_grid, kThreads,
                            sizeof(PersistSmem<false>), s, pa);
    else if (small)
      e = vals ? launch_pdl(onesweep_kernel<kItemsSmall, true>, (unsigned)parts, kThreads,
                            sizeof(PassSmem<kItemsSmall>), s, pa)
               : launch_pdl(onesweep_kernel<kItemsSmall, false>, (unsigned)parts, kThreads,
                            sizeof(PassSmem<kItemsSmall>), s, pa);
    else
      e = vals ? launch_pdl(onesweep_kernel<kItemsLarge, true>, (unsigned)parts, kThreads,
                            sizeof(PassSmem<kItemsLarge>), s, pa)
               : launch_pdl(onesweep_kernel<kItemsLarge, false>, (unsigned)parts, kThreads,
                            sizeof(PassSmem<kItemsLarge>), s, pa);
    if (e != cudaSuccess) return e;
    unsigned long long* tk = kin; kin = kout; kout = tk;
    uint32_t* tv = vin; vin = vout; vout = tv;
  }
  *result_in_alt = (passes & 1) != 0;
  if (sel) {
    *result_in_alt = false;
    *result_sel = sel + passes;
  }
  return cudaSuccess;
}

}  // namespace fs4d

// ---------------------------------------------------------------- allocation-free variant
// fs4d_sort_pairs_noalloc runs the same sort with every scratch buffer (the
// alternate key/value buffers, the digit histograms, the partition tickets, the
// look-back table and the status word) carved out of one file-scope device
// array, so the call itself never allocates.
#include <mutex>

namespace fs4d {
namespace {

constexpr long long kNaMaxPairs = FS4D_NOALLOC_MAX_PAIRS;
constexpr long long kNaParts = (kNaMaxPairs + kPartPairs - 1) / kPartPairs;
constexpr size_t kNaKeys = 0;
constexpr size_t kNaValues = kNaKeys + 8 * (size_t)kNaMaxPairs;
constexpr size_t kNaHist = kNaValues + 4 * (size_t)kNaMaxPairs;
constexpr size_t kNaCounters = kNaHist + 4 * (size_t)kMaxPasses * kRadix;
constexpr size_t kNaStatus = kNaCounters + 4 * (size_t)(2 * kMaxPasses + 1);  // tickets + selection words
constexpr size_t kNaLookback = (kNaStatus + 4 + 255) / 256 * 256;
constexpr size_t kNaBytes = kNaLookback + 4 * (size_t)kMaxPasses * kNaParts * kRadix;
constexpr int kNaMaxDevices = 64;

// The work area itself.  In host code this name is only a stand-in: its device
// address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_sort_scratch[kNaBytes];

std::mutex g_na_mutex;
unsigned char* g_na_base[kNaMaxDevices] = {};

// Device address of the work area on the current device (looked up once per device).
fs4d_status na_base(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return FS4D_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_base[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return FS4D_ERR_CUDA;
    g_na_base[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_na_base[dev];
  return FS4D_OK;
}

}  // namespace
}  // namespace fs4d

extern "C" fs4d_status fs4d_sort_pairs_noalloc(void* cuda_stream, int64_t n, int32_t key_bits, uint64_t* d_keys,
                                               uint32_t* d_values) {
  using namespace fs4d;
  if (n < 0 || key_bits < 1 || key_bits > 64 || (n > 0 && (!d_keys || !d_values))) return FS4D_ERR_INVALID_ARG;
  if (n > kNaMaxPairs) return FS4D_ERR_CAPACITY;
  if (n == 0) return FS4D_OK;
  unsigned char* base = nullptr;
  const fs4d_status bs = na_base(&base);
  if (bs != FS4D_OK) return bs;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  uint32_t* status = reinterpret_cast<uint32_t*>(base + kNaStatus);
  if (cudaMemsetAsync(status, 0, 4, s) != cudaSuccess) return FS4D_ERR_CUDA;
  SortWork w;
  w.hist = reinterpret_cast<uint32_t*>(base + kNaHist);
  w.lookback = reinterpret_cast<uint32_t*>(base + kNaLookback);
  w.part_counters = reinterpret_cast<uint32_t*>(base + kNaCounters);
  w.max_parts = kNaParts;
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(d_keys);
  unsigned long long* keys_alt = reinterpret_cast<unsigned long long*>(base + kNaKeys);
  uint32_t* values_alt = reinterpret_cast<uint32_t*>(base + kNaValues);
  bool alt = false;
  if (launch_sort(keys, d_values, keys_alt, values_alt, nullptr, n, 0, key_bits, false, w, status, s, &alt,
                  nullptr) != cudaSuccess)
    return FS4D_ERR_CUDA;
  if (alt) {
    if (cudaMemcpyAsync(d_keys, keys_alt, 8 * (size_t)n, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_values, values_alt, 4 * (size_t)n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return FS4D_ERR_CUDA;
  }
  return FS4D_OK;
}

extern "C" fs4d_status fs4d_sort_pairs_noalloc_status(void* cuda_stream, uint32_t* out) {
  using namespace fs4d;
  if (!out) return FS4D_ERR_INVALID_ARG;
  unsigned char* base = nullptr;
  const fs4d_status bs = na_base(&base);
  if (bs != FS4D_OK) return bs;
  if (cudaMemcpyAsync(out, base + kNaStatus, 4, cudaMemcpyDefault, reinterpret_cast<cudaStream_t>(cuda_stream)) !=
      cudaSuccess)
    return FS4D_ERR_CUDA;
  return FS4D_OK;
}
