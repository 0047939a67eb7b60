// Tensor-memory-accelerator (TMA) tile loads for the FP32 step: one thread issues a 3-D bulk tensor copy
// (x, y, conserved component) of the tile's padded box from global into shared memory, completion is
// signalled on a shared-memory mbarrier, and every thread waits on it with a bounded number of polls.
// PTX forms: cp.async.bulk.tensor (3-D, tile mode, mbarrier::complete_tx), mbarrier.init / arrive.expect_tx
// / try_wait.parity (PTX ISA 8.x, sm_90 and later).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hydro {

// polls of the mbarrier before a copy is declared lost (each poll may suspend the thread for a
// hardware-chosen time; a copy normally lands within a few microseconds)
constexpr unsigned int TMA_WAIT_POLLS = 1u << 22;

__device__ __forceinline__ unsigned int smem_addr(const void* p) {
  return static_cast<unsigned int>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned int bar, unsigned int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned int bar, unsigned int bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_inval(unsigned int bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before later async-proxy (TMA) ones.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bounded wait (polls polls) for the phase with the given parity to complete; true if it did.
__device__ __forceinline__ bool mbar_wait(unsigned int bar, unsigned int parity, unsigned int polls) {
  for (unsigned int k = 0; k < polls; ++k) {
    unsigned int done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// 3-D tile load: box at coordinates (x, y, z) of the tensor described by *map into shared memory at dst,
// completing `bytes` of transaction on bar.  x * element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_3d(unsigned int dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned int bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

}  // namespace hydro
