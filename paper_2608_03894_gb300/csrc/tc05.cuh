// Fifth-generation tensor-core helpers (sm_100 family, inline PTX): the
// shared-memory matrix descriptor of the 32-byte-swizzled K-major tiles the
// digit-slice kernels use, tcgen05.mma with a tensor-memory accumulator,
// tcgen05.commit / tcgen05.ld, bulk asynchronous copies (cp.async.bulk)
// completing on an mbarrier, and bounded mbarrier waits.
//
// Operand tiles: rows of 16 bf16 positions (32 bytes) along K; in every group
// of 8 rows, rows 4..7 have their two 16-byte halves swapped (the 32-byte
// swizzle), so element (v, k) of a tile sits at bf16 index
//     v * 16 + ((((k >> 3) ^ (v >> 2)) & 1) << 3) + (k & 7).
// A tile starts on a 256-byte boundary.
#pragma once

#include <stdint.h>

namespace dq {
namespace tc5 {

constexpr int kWaitLimit = 1 << 26;  // polls of a bounded wait (~0.1-1 s)

// bf16 index of element (v, k < 16) inside a swizzled tile
__host__ __device__ __forceinline__ int swz(int v, int k) {
  return v * 16 + ((((k >> 3) ^ (v >> 2)) & 1) << 3) + (k & 7);
}

// instruction descriptor of kind::f16 with bf16 operands, FP32 accumulator,
// both operands K-major, an M x N tile
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// shared-memory matrix descriptor of a swizzled tile: start address, leading
// byte offset 16 (unused: one K = 16 step is the whole row), stride byte
// offset 256 (8-row groups), version 1, layout type 6 (32-byte swizzle)
__device__ __forceinline__ uint64_t desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(16 >> 4) << 16) |
         ((uint64_t)(256 >> 4) << 32) | (1ull << 46) | (6ull << 61);
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of
// 16) completing `bytes` of transaction count on the mbarrier
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}
// Bounded wait for the phase with the given parity, polling with the
// non-blocking test (try_wait may suspend the thread for a system-dependent
// time, which would add its wake-up latency to every hand-over). Gives up
// when another role has raised *abort, or after kWaitLimit polls, when it
// raises *abort itself; returns whether the phase completed.
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t addr, uint32_t parity, volatile int *abort) {
  for (int it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.test_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.b32 %0, 1, 0, P;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 1023) == 1023 && *abort) return false;
  }
  *abort = 1;
  return false;
}
// Bounded wait that suspends the thread in hardware (mbarrier.try_wait with
// a suspend-time hint: the thread resumes when the phase completes, or after
// the hint) instead of spinning, for a wait of many cycles (a whole copy or
// MMA batch) whose issue slots other warps of the SM need. Gives up when
// *abort is raised or after kSleepWaitCycles clock cycles (~0.5 s), raising
// *abort itself.
constexpr long long kSleepWaitCycles = 1ll << 30;
constexpr uint32_t kSuspendHintNs = 100000;  // a suspended thread resumes when the phase completes
__device__ __forceinline__ bool mbar_sleep_wait(uint32_t addr, uint32_t parity, volatile int *abort) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, %3;\n selp.b32 %0, 1, 0, P;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity), "r"(kSuspendHintNs)
        : "memory");
    if (ok) return true;
    if (*abort) return false;
    if (clock64() - t0 > kSleepWaitCycles) {
      *abort = 1;
      return false;
    }
  }
}
// D (tensor memory) = A B^T (+ D when acc != 0), A and B from shared memory
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}
// arrive on the mbarrier when every MMA issued so far by this thread is done
__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
// tensor-memory allocation by one whole warp; the address lands in *slot
__device__ __forceinline__ void alloc(uint32_t *slot, int cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
               "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
}
__device__ __forceinline__ void dealloc(uint32_t taddr, int cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(cols));
}
// 8 / 16 columns of this warp's 32 lanes into v; the caller waits (wait_ld)
__device__ __forceinline__ void ld8(uint32_t taddr, float *v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc5
}  // namespace dq
