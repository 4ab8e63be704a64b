// Device side of the per-launch timestamps (see sy_internal.h): the first
// thread of every block records its start and, after the block's last store,
// its end and completion.  `s` is a kernel argument (uniform), so the barrier
// inside the branch is reached by every thread of the block or by none.
#pragma once

#include <cstdint>

namespace sy {

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void stamp_begin(unsigned long long* s) {
    if (s != nullptr && threadIdx.x == 0) atomicMax(&s[0], ~globaltimer_ns());
}

__device__ __forceinline__ void stamp_end(unsigned long long* s) {
    if (s != nullptr) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicMax(&s[1], globaltimer_ns());
            atomicAdd(&s[2], 1ull);
        }
    }
}

// Programmatic dependent launch (griddepcontrol): a kernel launched with the
// programmatic-stream-serialisation attribute may start while its predecessor on
// the stream is still running.  wait blocks until the predecessor grid has
// completed and its writes are visible (it returns at once for a kernel launched
// without the attribute); launch_dependents lets the next such kernel launch.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

}  // namespace sy
