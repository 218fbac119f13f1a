// Multi-source shortest paths in 32-source chunks (sssp.cu).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include "cc_internal.h"

namespace ccg {

constexpr int kChunkSrc = 32;  // sources per chunk: one 128-byte row per node

struct SsspJob {
    int64_t n;
    const int64_t *rp;
    const int32_t *col;
    const uint32_t *w;      // arc lengths (NULL: unit lengths)
    int kc;                 // sources in this chunk (<= 32 spl)
    int spl;                // sources per lane: 1 (rows of 32) or 2 (rows of 64)
    const int32_t *sources; // kc node ids
    uint32_t *dist;         // n x 32 spl
    unsigned long long *mask;  // n: sources whose distance dropped
    int32_t *Q0, *Q1;       // n each
    // Buckets (delta-stepping with a near and a far queue): labels below the
    // threshold T relax in rounds; labels at or beyond it wait in far queues
    // until the near queue empties and T grows by delta (0: no buckets, T
    // infinite).
    uint64_t delta;
    int32_t *far[3];        // n each
    uint32_t *nstamp, *fstamp;  // n each: round / epoch a node was last queued for
    Ctl *ctl;
    uint64_t timeout_ns;
    int max_ctas;           // 0: a whole-GPU launch
};

struct ReduceJob {
    int64_t n;
    int k, kc, base, W;
    int sum_only;                   // exact mode: only sum2 and the reachability check
    const uint32_t *distF, *distR;  // n x ld each (distR NULL unless round trip)
    const int32_t *row_of;          // row of node v (NULL: row v)
    int ld, sub;                    // row stride; this job's first column
    const int32_t *sidx;
    uint64_t *sum2;                 // n x 2
    unsigned long long *best;       // n: (distance << 32 | sample index) minimum
    uint32_t *dcc;                  // k x k
    unsigned long long *S_samp;     // k
    unsigned long long *dmax;       // 1
    int *err;                       // 1
    uint32_t *hist;                 // (D+1) x k
    int64_t D;                      // largest distance (hist has D+1 rows)
    const uint64_t *Lmask;          // n x W
    uint64_t *lc2;                  // n x 2
    // error estimate (null sqflag: not wanted): per node flag 1 adds
    // (d(c_i, v) - d(c(v), c_i))^2 over c_i outside Lmask into the 128-bit
    // hcse[v] = {lo, hi}; flag 2 records fdist[v] = d(c_i, v) for
    // c_i = istar[c(v)]
    const uint8_t *sqflag;
    const int32_t *istar, *pivot;
    uint64_t *hcse;                 // n x 2
    uint32_t *fdist;                // n
};

int launch_mssp(const SsspJob &job, cudaStream_t st);
void run_reduce1(const ReduceJob &r, cudaStream_t st);
void run_reduce2(const ReduceJob &r, cudaStream_t st);
void run_unpack_pivot(int64_t n, const unsigned long long *best, int32_t *pivot,
                      uint32_t *delta, cudaStream_t st);

}  // namespace ccg
