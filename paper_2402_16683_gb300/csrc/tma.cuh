// Bulk tensor copies (TMA) into shared memory, completing on an mbarrier.
//
// Tensor maps cover buffers of this device only and are never multicast.  A
// tiled load must start at an innermost coordinate whose byte offset is a
// multiple of 16; callers round x down and index from the remainder.  Every
// wait on an mbarrier is bounded: after the limit the waiter records a timeout
// in a status word that the host reads, and the kernel skips its remaining
// work (after waiting, again bounded, for its copies in flight).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace nre {

// Tiled tensor map of a row-major array: dims[0] innermost (elements),
// strides_b[d] the byte stride of dimension d + 1 (multiples of 16), box[d]
// the copied extent (box[0] * element size a multiple of 16, each <= 256).
// Out-of-range elements of a box read as zero.
int tmap_tiled(CUtensorMap* m, CUtensorMapDataType dt, int rank, const void* base, const uint64_t* dims,
               const uint64_t* strides_b, const uint32_t* box, int swizzle_bytes = 0);
// swizzle_bytes 32 / 64 / 128: the box's rows of that many bytes are stored in
// shared memory with their 16-byte chunks permuted: byte address A holds what
// the unswizzled layout has at A ^ ((A >> 3) & mask), mask 0x10 / 0x30 / 0x70
// (the box must start at a multiple of 1024 bytes).

// Per-device count of waits that ran out (allocated on first use; call it once
// outside stream capture, e.g. when a plan is created).
unsigned* timeout_word();

// Iterations of a bounded mbarrier wait (each try_wait suspends for a
// hardware-chosen time slice): about a second on a GB300 before giving up.
constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Make the initialised barriers visible to the async proxy (TMA).
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
// Order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (TMA) accesses of it.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Arrive on the barrier and announce `bytes` of transactions for this phase.
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bounded wait for the phase of the given parity; false after `limit` tries.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned limit = kWaitLimit) {
  const unsigned a = smem_u32(bar);
  for (unsigned it = 0; it < limit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* m, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* m, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* m, int x, int y, int z, int w,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}

// Bulk copy of `bytes` contiguous bytes (both addresses 16-byte aligned, a
// multiple of 16 bytes) from global memory to the shared address dst,
// completing on the mbarrier at shared address bar.
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// mbar_arrive_tx on the barrier at shared address bar.
__device__ __forceinline__ void mbar_arrive_tx_at(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

// Bulk tensor store of a box from shared memory (this thread's bulk group).
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* m, int x, int y, int z, int w, const void* src) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];\n" ::"l"(
                   reinterpret_cast<uint64_t>(m)),
               "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// Wait until this thread's committed bulk stores have read their shared
// memory (.read) or completed.
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// Record a wait that ran out (status[0] counts them).
__device__ __forceinline__ void note_timeout(unsigned* status) {
  if (status) atomicAdd(status, 1u);
}

}  // namespace nre
