// Tensor-memory-accelerator (TMA) tile loads with mbarrier completion.
//
// Host: tensor maps of this GPU's own device buffers, encoded with the driver's
// cuTensorMapEncodeTiled (reached through the runtime's entry-point query, so
// the library does not link libcuda).  Device: mbarrier initialisation,
// expect-tx arrival, bounded parity waits, and cp.async.bulk.tensor loads of
// 3D boxes into shared memory.  No multicast: every load is issued by the CTA
// that consumes it.
//
// Every wait is bounded: after kWaitLimit polls it gives up and reports
// failure, so a kernel never spins forever; callers record the timeout in
// g_tma_timeouts and turn their results into NaN, which the host sees as a
// failed solve.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace apfc {

// ---- host ------------------------------------------------------------------------
// Encode a rank-3 tiled tensor map over FP64 data: dims[0] is the innermost
// extent in doubles, strides[0..1] the byte strides of dims 1 and 2, box[0..2]
// the box extent (box[0] * 8 must be a multiple of 16).  Out-of-range box
// elements read as zero.  Returns false (with a message) if the driver has no
// TMA or rejects the arguments.
bool tma_encode_f64(CUtensorMap* map, const void* base, const unsigned long long dims[3],
                    const unsigned long long strides[2], const unsigned box[3], const char** err);
// The same with rank 4 (strides[0..2]: byte strides of dims 1..3).
bool tma_encode_f64_4d(CUtensorMap* map, const void* base, const unsigned long long dims[4],
                       const unsigned long long strides[3], const unsigned box[4], const char** err);

// Rank-4 tiled tensor map of any element type (box[0] * element bytes a multiple of 16).
bool tma_encode_4d(CUtensorMap* map, CUtensorMapDataType type, const void* base, const unsigned long long dims[4],
                   const unsigned long long strides[3], const unsigned box[4], const char** err);

// Number of TMA waits that timed out since the library was loaded (all devices).
unsigned long long tma_timeouts();

// ---- device ------------------------------------------------------------------------
constexpr unsigned kWaitLimit = 1u << 24;  // polls of one bounded wait (about a second)

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make the initialised barriers visible to the async proxy (TMA)
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// order this thread's generic-proxy shared-memory accesses before later async-proxy ones
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Wait for the phase of the given parity to complete; false after kWaitLimit polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  const unsigned a = smem_u32(bar);
  for (unsigned it = 0; it < kWaitLimit; ++it) {
    unsigned done;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 3D tiled box load global -> shared, completing on bar (coordinates in elements,
// innermost first; x * 8 bytes must be a multiple of 16).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, unsigned long long* bar, int x, int y,
                                            int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// 4D tiled box load (coordinates innermost first; x * 8 bytes a multiple of 16).
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, unsigned long long* bar, int x, int y,
                                            int z, int w) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<unsigned long long>(map)) : "memory");
}

}  // namespace apfc
