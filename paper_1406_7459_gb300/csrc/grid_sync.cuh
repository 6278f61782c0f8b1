// grid_sync.cuh -- a bounded grid-wide barrier for cooperative launches,
// and a work queue of tiles for persistent kernels.
//
// The barrier is an arrival counter in global memory that grows through
// the launch: barrier k is passed when (k + 1) x gridDim.x blocks have
// arrived.  Waits poll with a short sleep and give up after a poll limit
// chosen per launch; a block whose wait gave up reports it (the caller sets
// its status bit) and leaves, and the other blocks then give up at their
// next barrier.  The last block to leave clears the counters (grid_exit),
// so the next launch starts clean even after a timeout.  Every block of the
// launch must be co-resident (cooperative launch attribute).
#pragma once
#include <cuda_runtime.h>

namespace mmk {

// Counters of the grid barrier and of the work queues (zeroed at
// creation; cleared again by the last block of every launch).
struct GridBar {
    unsigned count;        // arrivals in this launch (every block once per barrier)
    unsigned exits;        // blocks that have left the launch
    unsigned queue[4];     // tiles taken from each work queue in this launch
    unsigned pad[2];
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier number `k` (0, 1, 2, ... within the launch): every block of the
// grid arrives before any proceeds; the writes of every thread before it are
// visible to every thread after it.  Each block adds 1 to the launch's
// arrival count and waits for it to reach (k + 1) blocks; the waits poll
// with a short sleep so that the arrivals are not slowed by the polls.
// Returns false, uniformly over the block, when its wait ran out of polls
// (limit 0: gives up at once unless every block has already arrived).
__device__ __forceinline__ bool grid_sync(GridBar* gb, unsigned k, long long limit) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        const unsigned target = (k + 1) * gridDim.x;
        __threadfence();
        red_release_add(&gb->count, 1u);
        long long it = 0;
        while ((int)(ld_acquire_gpu(&gb->count) - target) < 0) {
            if (it++ >= limit) {
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
}

// Last act of every block: the last one out clears the counters for the
// next launch.
__device__ __forceinline__ void grid_exit(GridBar* gb) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&gb->exits, 1u) == gridDim.x - 1) {
            atomicExch(&gb->count, 0u);
            for (int q = 0; q < 4; ++q) atomicExch(&gb->queue[q], 0u);
            atomicExch(&gb->exits, 0u);
        }
    }
}

// Next tile of work queue q for this block, or -1 when the queue is empty.
// Every block takes tiles until it meets an empty queue, so the queue's
// counter grows by exactly tiles + gridDim.x per pass over it; `round`
// counts the passes before this one in the launch.  The same tile never
// goes to two blocks.
__device__ __forceinline__ int queue_next(GridBar* gb, int q, int tiles, unsigned round, int* slot) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned base = round * (unsigned)(tiles + gridDim.x);
        const int i = (int)(atomicAdd(&gb->queue[q], 1u) - base);
        *slot = i < tiles ? i : -1;
    }
    __syncthreads();
    return *slot;
}

}  // namespace mmk
