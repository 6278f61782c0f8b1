// bulk_copy.cuh -- bulk asynchronous copies global -> shared memory through
// the tensor memory accelerator (cp.async.bulk), completed on an mbarrier,
// with bounded waits.
//
// One elected thread initialises an mbarrier (arrival count 1), announces the
// number of bytes it will deliver (arrive.expect_tx) and issues contiguous
// copies whose completion is counted on that barrier; every thread that
// reads the data waits on the barrier's phase 0.  A copy needs 16-byte
// aligned source and destination and a size that is a multiple of 16 bytes.
//
// Waits are bounded (kBulkWaitLimit polls, well under a second): a wait that
// runs out returns false, the kernel records kFlagTimeout in its status
// word, waits once more (again bounded) for its copies in flight, so that no
// copy lands in shared memory after the block has left, and returns.
#pragma once
#include <cuda.h>   // CUtensorMap (the type only; maps are encoded on the host)
#include <cuda_runtime.h>

#include <cstdint>

namespace mmk {

// Bits of the device status word (the context's flag): a non-finite state,
// a device wait that gave up.
constexpr int kFlagNonFinite = 1;
constexpr int kFlagTimeout = 2;

constexpr long long kBulkWaitLimit = 1LL << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Make initialised barriers visible to the async proxy and other threads
// (followed by a block barrier in the caller).
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Arrive once and expect `bytes` of transactions on the barrier's phase.
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Contiguous copy of `bytes` from global `src` to shared `dst`, counted on `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Order this thread's earlier generic-proxy view of global memory (data other
// threads wrote with ordinary stores and that this thread has synchronised
// with) before its following bulk copies read it.
__device__ __forceinline__ void proxy_fence_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
// The same for shared memory that the block has accessed with ordinary loads
// and stores (after a block barrier) and that bulk copies overwrite next.
__device__ __forceinline__ void proxy_fence_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Tiled tensor copies (cp.async.bulk.tensor) through a tensor map that is
// a __grid_constant__ kernel parameter.  The shared-memory side is the box
// of the map, innermost dimension fastest, starting on 128 bytes; the
// innermost coordinate times the element size is a multiple of 16 bytes.
__device__ __forceinline__ void tensor_prefetch(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}

// 4-D box at (x0, x1, x2, x3) from global memory to shared `dst`, counted on `bar`.
__device__ __forceinline__ void tensor_g2s_4d(uint32_t dst, const CUtensorMap* map, int x0, int x1, int x2, int x3,
                                              uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(map), "r"(x0), "r"(x1), "r"(x2), "r"(x3), "r"(bar)
        : "memory");
}

// 4-D box from shared `src` to global memory at (x0, x1, x2, x3), in this
// thread's current bulk group (bulk_commit, then bulk_wait_all before the
// shared memory is reused or the block leaves).
__device__ __forceinline__ void tensor_s2g_4d(const CUtensorMap* map, int x0, int x1, int x2, int x3, uint32_t src) {
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(map),
                 "r"(x0), "r"(x1), "r"(x2), "r"(x3), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Completion (writes done) of every bulk group this thread committed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Bounded wait for the phase of parity `parity` of `bar` to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long it = 0; it < kBulkWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace mmk
