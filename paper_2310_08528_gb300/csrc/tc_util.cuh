// tcgen05 building blocks shared by the BF16 tensor-core kernels (the deformation
// MLP and the colour/opacity heads): shared-memory operand descriptors in the UMMA
// canonical no-swizzle K-major layout, the instruction descriptor of kind::f16
// (BF16 x BF16 -> FP32), single-thread MMA issue with an mbarrier commit, bounded
// mbarrier waits, TMEM allocation and 32-lane accumulator loads.  M is 128 rows
// (one TMEM lane per row) throughout.
#pragma once

#include "fs4d_internal.cuh"

namespace fs4d {
namespace tcu {

constexpr int kTcRows = 128;
constexpr uint32_t kWaitLimit = 1u << 20;  // mbarrier polls before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start address, LBO = byte
// distance between core matrices along K, SBO = along M/N, version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor: kind::f16, A = B = BF16, D = F32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// one arrival (release, CTA scope) on an mbarrier initialised with count 1
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
// barrier `id` (1..15) of `n` threads (a multiple of 32): one warp group's __syncthreads
__device__ __forceinline__ void group_sync(uint32_t id, uint32_t n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// group_sync that also ORs `pred` over the group: the same answer in every thread
__device__ __forceinline__ bool group_sync_or(uint32_t id, uint32_t n, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 lanes x 32 columns of FP32 (this warp's lane quarter), waited on in the same asm.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (r, k) in a K-major no-swizzle operand with K columns:
// 8x8 core matrices of 128 contiguous bytes, (r/8, k/8) at ((r/8)*(K/8) + k/8)*128.
__device__ __forceinline__ uint32_t a_off(int r, int k, int K) {
  return (uint32_t)(((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// relu(v + bias) of 32 columns -> BF16 row segment k0..k0+31 of an operand with K columns.
__device__ __forceinline__ void store_relu32(uint8_t* tile, int r, int k0, int K, const float (&v)[32],
                                             const float* bias) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint4 q;
    q.x = pack_bf16(fmaxf(v[8 * j + 0] + bias[8 * j + 0], 0.f), fmaxf(v[8 * j + 1] + bias[8 * j + 1], 0.f));
    q.y = pack_bf16(fmaxf(v[8 * j + 2] + bias[8 * j + 2], 0.f), fmaxf(v[8 * j + 3] + bias[8 * j + 3], 0.f));
    q.z = pack_bf16(fmaxf(v[8 * j + 4] + bias[8 * j + 4], 0.f), fmaxf(v[8 * j + 5] + bias[8 * j + 5], 0.f));
    q.w = pack_bf16(fmaxf(v[8 * j + 6] + bias[8 * j + 6], 0.f), fmaxf(v[8 * j + 7] + bias[8 * j + 7], 0.f));
    *reinterpret_cast<uint4*>(tile + a_off(r, k0 + 8 * j, K)) = q;
  }
}

// The MMAs of a GEMM over columns [k0, k0 + kn) of two K-major operands with K
// columns (k0, kn multiples of 16) into TMEM column `col`; no commit.
__device__ __forceinline__ void issue_mmas(uint32_t tmem, int col, uint32_t a_addr, uint32_t b_addr, int K, int k0,
                                           int kn, int N) {
  const uint32_t sbo = (uint32_t)(K / 8) * 128u;
  const uint32_t id = idesc_bf16(kTcRows, N);
  for (int kk = 0; kk < kn / 16; ++kk) {
    const uint32_t off = 256u * (uint32_t)(k0 / 16 + kk);
    const uint64_t da = smem_desc(a_addr + off, 128u, sbo);
    const uint64_t db = smem_desc(b_addr + off, 128u, sbo);
    mma(tmem + (uint32_t)col, da, db, id, kk > 0 ? 1u : 0u);
  }
}

// One GEMM of K columns into TMEM column `col`: K/16 MMAs, then a commit.
__device__ __forceinline__ void issue_gemm(uint32_t tmem, int col, uint32_t a_addr, uint32_t b_addr, int K, int N,
                                           uint32_t mbar) {
  issue_mmas(tmem, col, a_addr, b_addr, K, 0, K, N);
  mma_commit(mbar);
}

}  // namespace tcu
}  // namespace fs4d
