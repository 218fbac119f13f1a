// Outbound / inbound reachability-sample estimates (reach.cu).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include "cc_internal.h"

namespace ccg {

constexpr int kReachMaxW = 16;  // words per node: groups of up to 1024 sources

struct ReachJob {
    int64_t n;
    int k, W;                     // sample size; words per node (1..kReachMaxW)
    const int64_t *rp;            // search graph (G^T: outbound, G: inbound)
    const int32_t *col;
    const uint32_t *w;            // its arc lengths (null: unit lengths)
    const int32_t *order, *rank;  // the random order and its inverse
    // per node
    int32_t *cnt;                 // samples taken (<= k)
    uint8_t *extra;               // a (k+1)-th source other than the node reached it
    uint64_t *dsum;               // sum of the samples' distances
    int64_t *T;                   // rank position of the k-th sample, mark rule
    uint32_t *qstamp;             // level stamp of the last push to the queue
    uint64_t *vis, *F, *nxt;      // n x W
    uint32_t *lev;                // n x 64 W: first-arrival level of each bit
                                  // (arc lengths: tentative distance, kInf
                                  // outside a group's search)
    int32_t *Q[2], *TL;           // frontier queues, touched list (n each)
    Ctl *ctl;                     // barrier counter and error code
    uint64_t timeout_ns;
};

struct ReachStats {
    int64_t levels, groups;
    int grid;
};

// order / rank (device, n each) of the seeded random order; scratch keys,
// tk (n uint64), vals, tv (n uint32).  Synchronises the stream.
int reach_order(int64_t n, uint64_t seed, uint64_t *keys, uint32_t *vals, uint64_t *tk,
                uint32_t *tv, int32_t *order, int32_t *rank, cudaStream_t st);

// The cooperative launch over every group; the per-node state must start
// zeroed.  Synchronises the stream; returns CC_ERR_TIMEOUT if a barrier wait
// ran out.
int reach_run(const ReachJob &job, cudaStream_t st, ReachStats *stats);

// avg = dsum / cnt (0 when cnt = 0); rhat = cnt when cnt < k, else
// 1 + (k-1)(n-2) / (T-1) (1 when k = 1).  Either output may be null.
void reach_finalize(int64_t n, int k, const int32_t *cnt, const uint64_t *dsum,
                    const int64_t *T, double *avg, double *rhat, cudaStream_t st);

}  // namespace ccg
