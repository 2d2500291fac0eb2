// Bulk asynchronous copies (cp.async.bulk, the TMA's untiled form) that
// complete on an mbarrier, with bounded waits: a copy that never lands
// makes the kernel record RTG_ERR_TIMEOUT and stop, never spin forever.
// Both addresses must be 16-byte aligned and the size a multiple of 16.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "rtg_internal.cuh"

namespace rtg {

// The driver's tensor-map encoder, looked up once (null if unavailable).
inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)));
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// An mbarrier that completes its phase after `count` plain arrivals.
__device__ __forceinline__ void mbar_init_n(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// One arrival (release semantics: this thread's earlier writes are visible
// to a thread whose wait observes the phase completing).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Every caller refills shared memory that its threads read with ordinary
// (generic-proxy) loads before the barrier that precedes the copy; the copy
// writes through the async proxy, so a proxy fence must order those reads
// before it.  Without the fence a copy can land before reads that the
// barrier has not yet performed -- observed as corrupted stretches of ring
// slots when CTAs of other kernels shared the SM (concurrent graph branches).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Tiled tensor copy (TMA, cp.async.bulk.tensor) of one box of a 3-D tensor
// map into shared memory, completing on an mbarrier.  tmap: the generic
// address of the map (a __grid_constant__ kernel parameter); c0: the
// innermost coordinate, whose byte offset must be a multiple of 16; boxes
// reaching past the tensor are filled with zeros.
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int c0, int c1, int c2, uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // as in bulk_g2s
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

// The same for a 5-D tensor map (coordinates innermost first).
__device__ __forceinline__ void tma_load_5d(void* dst, const void* tmap, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar) {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // as in bulk_g2s
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];\n" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
      : "memory");
}

// Bulk copy shared -> global (bulk-group completion); both addresses
// 16-byte aligned, size a multiple of 16.  The issuing thread commits the
// group and waits until the source has been read before the shared memory
// may be released or reused.
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_s2g_commit_and_wait_read() {
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}

// Waits for phase `parity`; gives up after a bounded number of polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Called by every thread after issuing a chunk's copies.  True if a copy
// did not land within the bounded wait (agreed across the CTA): thread 0
// then waits once more, bounded, for the copies still in flight, and the
// timeout is recorded in *status.  The caller stops issuing copies.
__device__ __forceinline__ bool tc_wait_failed(uint64_t* bar, uint32_t phase, int* status) {
  const bool landed = mbar_wait(bar, phase);
  if (!__syncthreads_or(!landed)) return false;
  if (threadIdx.x == 0) {
    mbar_wait(bar, phase);
    if (status != nullptr) atomicExch(status, RTG_ERR_TIMEOUT);
  }
  __syncthreads();
  return true;
}

}  // namespace rtg
