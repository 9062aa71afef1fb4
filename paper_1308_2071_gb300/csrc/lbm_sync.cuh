// Grid-wide synchronisation for persistent kernels (cooperative launches,
// every block resident): a bounded barrier, so that a block that waits too
// long records a timeout and returns instead of hanging the GPU.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

// Bounded sense-reversing grid barrier.  Thread 0 of each block arrives on
// count; the last arrival resets count and bumps gen; the others wait for gen
// to change, at most `limit` polls (sleeps growing from 32 ns to max_ns).
// Returns false (in every thread of the block) when the wait ran out, after
// setting bit 0 of *flag.
__device__ __forceinline__ bool grid_barrier(unsigned* count, volatile unsigned* gen, unsigned nblocks,
                                             long long limit, int* flag, int* reset_on_release,
                                             unsigned max_ns = 1024) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(count, 0u);
            if (reset_on_release) atomicExch(reset_on_release, 0);
            __threadfence();
            atomicAdd((unsigned*)gen, 1u);
        } else {
            long long polls = 0;
            unsigned ns = 32;  // exponential back-off keeps thousands of pollers off the L2 slice
            while (*gen == g) {
                if (++polls > limit) {
                    ok = 0;
                    atomicOr(flag, 1);
                    break;
                }
                __nanosleep(ns);
                ns = ns < max_ns ? 2 * ns : max_ns;
            }
        }
        __threadfence();
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

}  // namespace lbm
