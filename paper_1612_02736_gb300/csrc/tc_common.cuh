// Device helpers shared by tcgen05 kernels: shared-memory addresses, the UMMA shared-memory
// descriptor of a K-major operand without swizzle, mbarrier waits with an iteration bound,
// asynchronous copies.  Every wait here is bounded: a wait that runs out sets the CTA's
// abort flag and the caller's status word (-1), and every role then stops.
#pragma once

#include <cstdint>

namespace hps {
namespace tc {

constexpr long long kWaitLimit = 1ll << 26;  // polls before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start address, leading-dimension byte offset
// (between the two 8-element halves of a 16-element K slice) and stride byte offset
// (between 8-row groups), no swizzle, fixed field 1 at bit 46.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Byte offset of (row, k) in a K-major plane of 16-bit elements with 16 k per row: 8-row x
// 16-byte core matrices, 128 bytes between the two k halves, 256 bytes between row groups.
__device__ __forceinline__ int kmaj(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ void mb_init(unsigned long long* b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ void mb_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mb_try(unsigned long long* b, int parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false on timeout (which raises the abort
// flag and sets *status = -1) or when another role has aborted.
__device__ __forceinline__ bool mb_wait(unsigned long long* b, int parity, volatile int* abort_flag, int* status) {
  for (long long it = 0; it < kWaitLimit; ++it) {
    if (mb_try(b, parity)) return true;
    if ((it & 255) == 255 && *abort_flag) return false;
  }
  *abort_flag = 1;
  if (status) atomicCAS(status, 0, -1);
  return false;
}
// The same wait with a caller-given poll limit.
__device__ __forceinline__ bool mb_wait_n(unsigned long long* b, int parity, long long limit, volatile int* abort_flag,
                                          int* status) {
  for (long long it = 0; it < limit; ++it) {
    if (mb_try(b, parity)) return true;
    if ((it & 255) == 255 && *abort_flag) return false;
  }
  *abort_flag = 1;
  if (status) atomicCAS(status, 0, -1);
  return false;
}
// Bounded wait that ignores the abort flag (a role draining its own operations at exit).
__device__ __forceinline__ void mb_drain(unsigned long long* b, int parity) {
  for (long long it = 0; it < kWaitLimit; ++it)
    if (mb_try(b, parity)) return;
}
// Warp-uniform bounded wait: lane 0 waits, the result is broadcast.
__device__ __forceinline__ bool warp_wait(unsigned long long* b, int parity, volatile int* abort_flag, int* status) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) ok = mb_wait(b, parity, abort_flag, status) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Arrive on the barrier and raise its expected transaction count by `bytes`.
__device__ __forceinline__ void mb_expect_arrive(unsigned long long* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
// Bulk copy (16-byte aligned addresses, size a multiple of 16) from global to shared memory
// that completes `bytes` transactions on the barrier.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace tc
}  // namespace hps
