// Relaxed GPU-scope loads/stores and a bounded spin used by the single-pass
// (decoupled look-back) kernels.  Every wait gives up after kSpinLimit polls,
// sets kStatusTimeout in the device status word and lets the kernel finish, so a
// lost predecessor can never hang the GPU.
#pragma once

#include "fs4d_internal.cuh"

namespace fs4d {

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t lane_id() {
  uint32_t l;
  asm volatile("mov.u32 %0, %%laneid;" : "=r"(l));
  return l;
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Lanes of the warp that hold the same digit as this lane (a warp multisplit from
// one ballot per digit bit; digits have `bits` <= 8 significant bits, the same in
// every lane); lanes with valid == false are in no lane's mask.  Every lane of
// the warp must call it.
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, bool valid, int bits = 8) {
  uint32_t m = __ballot_sync(0xffffffffu, valid);
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    if (b >= bits) break;  // warp-uniform
    const bool bit = (d >> b) & 1u;
    const uint32_t bal = __ballot_sync(0xffffffffu, bit);
    m &= bit ? bal : ~bal;
  }
  return m;
}

}  // namespace fs4d
