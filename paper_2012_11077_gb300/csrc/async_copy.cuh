// Asynchronous-copy and barrier helpers shared by the kernels (inline PTX):
// cp.async (LDGSTS) into shared memory, the bulk-copy engine
// (cp.async.bulk, completion counted in bytes on an mbarrier) and bounded
// mbarrier waits.
#pragma once

#include "rcfar_internal.cuh"

namespace rcfar {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// 16-byte cp.async; valid == false zero-fills the 16 bytes and reads nothing.
__device__ __forceinline__ void cp_async16(unsigned saddr, const void* gmem, bool valid) {
  const int src_bytes = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(gmem), "r"(src_bytes) : "memory");
}
// 4-byte cp.async through L1; valid == false zero-fills the 4 bytes and reads nothing.
__device__ __forceinline__ void cp_async4(unsigned saddr, const void* gmem, bool valid) {
  const int src_bytes = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(saddr), "l"(gmem), "r"(src_bytes) : "memory");
}
// 16-byte cp.async of src_bytes (0..16) bytes, the rest zero-filled; src
// and dst 16-byte aligned (src need not be read when src_bytes is 0).
__device__ __forceinline__ void cp_async16_n(unsigned saddr, const void* gmem, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(gmem), "r"(src_bytes) : "memory");
}
// Shared-memory accesses by 32-bit shared-window address.
__device__ __forceinline__ unsigned long long lds_u64(unsigned a) {
  unsigned long long v;
  asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts_u64(unsigned a, unsigned long long v) {
  asm volatile("st.shared.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
__device__ __forceinline__ float lds_f32(unsigned a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
// 8-byte cp.async through L1 (both addresses 8-byte aligned).
__device__ __forceinline__ void cp_async8(unsigned saddr, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(saddr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Order this thread's generic-proxy shared-memory writes before later
// async-proxy (bulk copy, tensor core) accesses of the same locations.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}
// Arrive once and add tx_bytes to the bytes the current phase waits for.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned tx_bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
               "r"(tx_bytes)
               : "memory");
}
// Wait for the phase of the given parity to complete; gives up after
// `limit` polls and returns false. Each poll may suspend the thread for up
// to kWaitHintNs until the phase completes, so waiting warps do not take
// issue slots from working ones.
constexpr unsigned kWaitHintNs = 1000;
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, unsigned limit) {
  for (unsigned it = 0; it < limit; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity), "n"(kWaitHintNs)
        : "memory");
    if (done) return true;
  }
  return false;
}
// The library's kernels wait at most kSpinLimit polls (about a second).
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  return mbar_wait_bounded(bar, parity, kSpinLimit);
}

// Bulk copy global -> shared of `bytes` (a multiple of 16; both addresses
// 16-byte aligned); completion is counted on the mbarrier in bytes.
__device__ __forceinline__ void bulk_g2s(unsigned saddr, const void* gmem, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(saddr),
               "l"(gmem), "r"(bytes), "r"(bar)
               : "memory");
}

// 3-D tiled tensor load global -> shared (box of the tensor map at
// coordinates {c0, c1, c2}, innermost first), completing on the mbarrier
// with its byte count; elements outside the tensor arrive as zeros.
// tmap: generic address of a CUtensorMap in param, const or global memory.
__device__ __forceinline__ void tma_load_3d(unsigned saddr, unsigned long long tmap, int c0, int c1, int c2,
                                            unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(saddr),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// 2-D tiled tensor load global -> shared (box at coordinates {c0, c1},
// innermost first), completing on the mbarrier with its byte count;
// elements outside the tensor arrive as zeros. c0 times the element size
// must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(unsigned saddr, unsigned long long tmap, int c0, int c1, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          saddr),
      "l"(tmap), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

}  // namespace rcfar
