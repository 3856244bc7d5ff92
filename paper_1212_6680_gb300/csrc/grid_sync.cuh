// grid_sync.cuh -- a bounded grid-wide barrier for kernels whose CTAs are all resident (a
// cooperative launch, or a persistent grid sized to the SMs): thread 0 of every CTA arrives on a
// counter; the last to arrive resets it and advances a generation word that the
// others poll.  The wait is bounded: after `limit` polls the waiter records SMG_ERR_TIMEOUT in
// *err and every CTA returns false, so a barrier that cannot complete ends the kernel with an
// error status instead of hanging.
#pragma once

#include "../../include/smg.h"

namespace smg {

__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned *gen, int *err, long long limit,
                                             unsigned expected) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = *reinterpret_cast<volatile unsigned *>(gen);
        __threadfence();
        const unsigned arrived = atomicAdd(count, 1u);
        if (arrived == expected - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            long long spins = 0;
            while (*reinterpret_cast<volatile unsigned *>(gen) == g) {
                if (*reinterpret_cast<volatile int *>(err) != 0) break;
                if (++spins > limit) {
                    atomicCAS(err, 0, SMG_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        ok = (*reinterpret_cast<volatile int *>(err) == 0);
    }
    __syncthreads();
    return ok != 0;
}

}  // namespace smg
