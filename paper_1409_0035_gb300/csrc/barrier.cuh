// Bounded barrier over the CTAs of a team (all co-resident: the kernels
// using it are cooperative launches).
//
// Thread 0 of every CTA adds 1 to the team's 64-bit arrival counter; since
// every CTA passes every barrier, the counter is a multiple of the team size
// between barriers, and the value a CTA's add returns tells which barrier it
// arrived at: it waits until the counter reaches the next multiple.  One
// atomic round trip per CTA and no resets (a two-level tree of counters with
// resets measured about 2.7 times slower on 608 CTAs).  A wait that runs past
// timeout_ns records CC_ERR_TIMEOUT, and every CTA stops waiting as soon as
// the team reports a negative error code.
#pragma once
#include <cstdint>

#include "cc_internal.h"

namespace ccg {
namespace {

__device__ __forceinline__ uint64_t bar_clock()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Returns false (in every thread of the CTA) when the wait ran out or the
// team reported an error.
__device__ bool grid_sync(Ctl *ctl, unsigned rank, unsigned nblocks, uint64_t timeout_ns)
{
    (void)rank;
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned long long *vc = &ctl->bar_arrive;
        volatile int *verr = &ctl->err;
        __threadfence();
        const unsigned long long old = atomicAdd(&ctl->bar_arrive, 1ull);
        const unsigned long long target = (old / nblocks + 1) * nblocks;
        if (*vc < target) {
            const uint64_t t0 = bar_clock();
            unsigned ns = 8;
            while (*vc < target) {
                if (*verr < 0) { ok = 0; break; }
                if (bar_clock() - t0 > timeout_ns) {
                    atomicCAS(&ctl->err, 0, CC_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(ns);
                if (ns < 64) ns <<= 1;
            }
        }
        __threadfence();
        if (*verr < 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Per-CTA staging of queue appends: appends go to shared memory and the
// CTA reserves its slots in the global queue with one atomicAdd when it
// flushes, instead of one global atomic per appended node.
constexpr int kStage = 1024;

struct Stage {
    int32_t *buf;      // shared, kStage entries
    unsigned *count;   // shared
    unsigned *base;    // shared
};

__device__ __forceinline__ void stage_push(const Stage &s, int32_t v, int32_t *gq,
                                           unsigned *glen)
{
    const unsigned p = atomicAdd(s.count, 1u);
    if (p < (unsigned)kStage) s.buf[p] = v;
    else gq[atomicAdd(glen, 1u)] = v;  // stage full: append directly
}

// Called by every thread of the CTA; leaves the stage empty.
__device__ __forceinline__ void stage_flush(const Stage &s, int32_t *gq, unsigned *glen)
{
    __syncthreads();
    const unsigned m = min(*s.count, (unsigned)kStage);
    if (threadIdx.x == 0) *s.base = m ? atomicAdd(glen, m) : 0u;
    __syncthreads();
    for (unsigned i = threadIdx.x; i < m; i += blockDim.x) gq[*s.base + i] = s.buf[i];
    __syncthreads();
    if (threadIdx.x == 0) *s.count = 0;
    __syncthreads();
}

}  // namespace
}  // namespace ccg
