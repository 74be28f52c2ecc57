// tma.cuh -- bulk copy-engine (TMA) staging of contiguous global ranges into
// shared memory, completed on an mbarrier (inline PTX, sm_90 and later).
//
// Protocol (one mbarrier per CTA, arrival count 1):
//   init once:  mbar_init(bar, 1); fence_mbar_init(); __syncthreads();
//   per use k:  after a block barrier that ends every generic access to the
//               destination, one thread runs fence_proxy_async(),
//               mbar_expect_tx(bar, total bytes) and the tma_load_1d copies;
//               readers call mbar_wait(bar, k & 1, ...) before touching the
//               destination.
// The wait is bounded: on time-out it records ADERDG_ETIMEOUT in the control
// block and returns false; every thread still reaches the same barriers.
#pragma once
#include "aderdg.h"
#include "common.cuh"

namespace aderdg {

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// orders this thread's (and, after a barrier, the block's) generic-proxy
// shared-memory accesses before later async-proxy (bulk copy) writes
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Bring a contiguous global range into L2 ahead of its loads (bulk copy engine,
// no completion tracking); src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void l2_prefetch_bulk(const void *src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// The same for a range of any alignment: only its 16-byte aligned interior is
// prefetched, so nothing outside [p, p + bytes) is touched.
__device__ __forceinline__ void l2_prefetch_range(const void *p, size_t bytes) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uintptr_t lo = (a + 15) & ~uintptr_t(15), hi = (a + bytes) & ~uintptr_t(15);
  if (hi > lo) l2_prefetch_bulk(reinterpret_cast<const void *>(lo), (unsigned)(hi - lo));
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with the given parity to complete; at most `limit`
// polls (each try_wait may suspend the thread for a hardware-chosen time).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, DevCtl *ctl,
                                          unsigned limit = 1u << 24) {
  for (unsigned i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicCAS(&ctl->error, 0, (int)ADERDG_ETIMEOUT);
  return false;
}

}  // namespace aderdg
