// Tensor-memory-accelerator (TMA) staging helpers for sm_100-class GPUs: shared-memory
// mbarriers with transaction counts, one-dimensional tiled bulk tensor copies from
// global into shared memory, and the host-side encoding of their tensor maps.
//
// A tensor map views a whole vector (u, E, the fixture mask, ...) as one row of n
// elements (a 2-D tensor n x 1).  A copy takes `box` consecutive elements starting at coordinate x (x *
// element size must be a multiple of 16 bytes); elements outside [0, n) arrive as
// zeros, so a tile's copies never read past an allocation.  Every wait is bounded:
// after kMbarSpins polls it records TO_ERR_TIMEOUT and returns false.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.cuh"

namespace to {

constexpr unsigned long long kMbarSpins = 1ull << 26;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make the initialised barriers visible to the async proxy (the TMA unit)
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// one arrival that also raises the phase's expected transaction bytes
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// wait for the completion of the phase with the given parity; bounded
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err) {
    for (unsigned long long i = 0; i < kMbarSpins; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    atomicCAS(err, 0, (int)TO_ERR_TIMEOUT);
    return false;
}

__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* m) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(m)) : "memory");
}

// box elements starting at x into shared memory at dst, completing on bar (the map is
// a one-row 2-D tensor: row coordinate 0)
__device__ __forceinline__ void tma_load_1d(void* dst, const CUtensorMap* m, int x, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(0), "r"(smem_u32(bar))
        : "memory");
}

// host: a 1-D tiled tensor map over n elements of `dtype` at `base` (16-byte aligned),
// copied `box` elements at a time (box * element size a multiple of 16, box <= 256)
int encode_map_1d(CUtensorMap* out, const void* base, unsigned long long n, CUtensorMapDataType dtype, unsigned esize,
                  unsigned box);

}  // namespace to
