// Bulk asynchronous copies global -> shared memory by the TMA engine (the 1D
// form cp.async.bulk, and 2D boxes of a tensor map, cp.async.bulk.tensor)
// completing on an mbarrier, with bounded waits.
//
// Rules these helpers rely on: source and destination 16-byte aligned, sizes a
// multiple of 16 bytes; one thread arms the barrier with the byte count of the
// copies of a phase (arrive.expect_tx) and issues them; consumers wait on the
// phase parity.  A wait gives up after a bounded number of polls and reports
// it, so a kernel never spins forever on a copy that does not land.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace mmc {

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make barrier initializations visible to the asynchronous proxy
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic-proxy accesses to shared memory before
// later asynchronous-proxy accesses (a buffer read by threads, then refilled by
// a bulk copy)
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// bytes (a multiple of 16) from global src to shared dst (both 16-byte aligned),
// counted on bar's transaction count
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// a 2D box of a tensor described by the tensor map at tmap (a kernel parameter
// declared __grid_constant__) from global to shared memory at coordinates
// (x, y) of the map (x in elements of the innermost dimension, x times the
// element size a multiple of 16 bytes); dst 128-byte aligned; counted on bar's
// transaction count
__device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// wait for the phase with the given parity; false if it did not complete within
// max_polls polls (each try_wait itself suspends the thread for a while)
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned max_polls) {
  for (unsigned i = 0; i < max_polls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

}  // namespace mmc
