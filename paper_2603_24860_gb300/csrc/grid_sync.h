// Bounded grid-wide barrier for cooperative launches (all CTAs co-resident)
// on sm_103a: one release-add per CTA on a counter and acquire-polling until
// it reaches the target.  Every wait is bounded: after `limit` polls (the
// default, kGridSpinLimit, is seconds of polling; a context can lower it, down
// to 0 = give up at once, to exercise the failure path), or when another CTA
// has raised the error flag, the barrier raises the flag and returns false so
// that the kernel can return.
#pragma once

#include <cuda_runtime.h>

namespace bse {

constexpr long kGridSpinLimit = 1l << 23;   // >= 32 ns + an L2 round trip per poll: seconds
constexpr long kMbarSpinLimit = 1l << 24;   // polls of an mbarrier wait (try_wait suspends in hardware): seconds

// the limit of a launch: the context's setting, or the default when it is negative
inline long wait_limit(long polls, long dflt) { return polls < 0 ? dflt : polls; }

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// target = (number of barriers so far) x gridDim.x; s_flag: a shared int of the CTA
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, int* err, int* s_flag,
                                             long limit = kGridSpinLimit) {
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
        bool ok = false;
        for (long it = 0; it < limit; ++it) {
            if (ld_acquire_gpu(bar) >= target) {
                ok = true;
                break;
            }
            if (*(volatile int*)err) break;
            if (it > 64) __nanosleep(32);
        }
        if (!ok) atomicExch(err, 1);
        *s_flag = ok ? 1 : 0;
    }
    __syncthreads();
    return *s_flag != 0;
}

}  // namespace bse
