// Bulk asynchronous copies (TMA, cp.async.bulk) and mbarriers for sm_100+,
// as inline PTX. Only 1-D bulk copies are used: global -> this CTA's own
// shared memory, 16-byte aligned addresses, sizes a multiple of 16 bytes. No
// tensor maps, no multicast, no clusters beyond the CTA itself.
//
// Every wait is bounded: try_wait is retried with a nanosleep back-off up to
// kWaitLimit times; a wait that gives up returns false and the caller records
// the failure in a device status word and leaves its loop.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hm {

// 2^20 polls with a back-off of up to 256 ns: a fraction of a second to a
// few seconds, far beyond any legitimate wait of a kernel whose whole run
// takes milliseconds.
constexpr unsigned kWaitLimit = 1u << 20;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// make the initialised barriers visible to the async proxy (the bulk copies)
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// one arrival plus `bytes` of expected transaction count
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete; false after the limit.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  // try_wait itself suspends the thread for a while in hardware: poll it
  // back to back first, and back off with sleeps only for a long wait
  for (int it = 0; it < 64; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  unsigned ns = 32;
  for (unsigned it = 0; it < kWaitLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    __nanosleep(ns);
    if (ns < 256) ns <<= 1;
  }
  return false;
}

// global -> shared bulk copy completing on `bar` (dst, src 16-byte aligned,
// bytes a positive multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

}  // namespace hm
