// Node-weighted closeness (section 5, "Weighted Centrality"): the weighted
// sampler and the weighted reductions over chunks of shortest-path rows
// (nodew.cu).  The orchestration lives in cc_api.cu.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace ccg {

// Sum of the weights (dsum: one device uint64 of scratch).  Synchronises.
int nw_total(const uint32_t *beta, int64_t n, uint64_t *dsum, uint64_t *total,
             cudaStream_t st);

// Threshold tau = tn / td of a weight vector (sum of min(1, beta/tau) = k),
// computed on the device into tau4[0..1] (tau4[2] = number of positive
// weights, tau4[3] scratch; tau = 0/0 when fewer than k weights are
// positive).  Scratch: keys, tk (n uint64), vals, tv (n uint32), pre (n
// uint64).  Synchronises the stream.
int nw_threshold(const uint32_t *beta, int64_t n, int k, uint64_t *keys, uint32_t *vals,
                 uint64_t *tk, uint32_t *tv, uint64_t *pre, uint64_t *tau4, cudaStream_t st);

// The nodes in increasing (splitmix64 output v of stream `seed`, v): a
// seeded random order, left in vals (in_tmp false) or tv (in_tmp true).
// Scratch: keys, tk (n uint64).  Synchronises the stream.
int random_order(int64_t n, uint64_t seed, uint64_t *keys, uint32_t *vals, uint64_t *tk,
                 uint32_t *tv, bool *in_tmp, cudaStream_t st);

// Systematic draw of the sample along the splitmix64 order of `seed` given tau
// (device): out[k] (device) receives the sampled nodes in that order; *count
// the number drawn (k by construction; entries past k are not written).  Scratch as nw_threshold, plus
// flags (n uint64).  Synchronises the stream.
int nw_draw(const uint32_t *beta, int64_t n, int k, uint64_t seed, const uint64_t *tau,
            uint64_t *keys, uint32_t *vals, uint64_t *tk, uint32_t *tv, uint64_t *pre,
            uint64_t *flags, int32_t *out, int64_t *count, cudaStream_t st);

// Per sampled node: bsrc[i] = beta(c_i), mu[i] = max(tau, beta(c_i)) * td
// (an integer: tn when beta(c_i) < tau, beta(c_i) td otherwise); msum[0] +=
// mu, msum[1] = 1 if some sampled node has weight 0.
void run_nw_mu(int k, const int32_t *sources, const uint32_t *beta, const uint64_t *tau,
               uint32_t *bsrc, uint64_t *mu, unsigned long long *msum, cudaStream_t st);

// One slice of at most 32 columns of the chunk's distance rows.
struct NwJob {
    int64_t n;
    int k, base, kc;
    const uint32_t *distF, *distR;  // n x ld each (distR null unless round trip)
    const int32_t *row_of;          // row of node v (null: row v)
    int ld, sub;                    // row stride; the slice's first column
    const uint32_t *beta;           // n
    const uint64_t *mu;             // k
    const uint32_t *bsrc;           // k
    const int32_t *sidx, *pivot;    // n
    const uint32_t *delta, *dcc;    // n; k x k
    uint64_t *wsum;                 // n: sum_i mu_i d(c_i, v)
    unsigned long long *S;          // k: sum_v beta(v) d(c_i, v)
    // second sweep (hybrid)
    uint32_t a, b;                  // eps = a / b
    unsigned long long *hist;       // (D + 1) x k: beta mass of V \ C per distance
    uint64_t *lc;                   // n x 2: {L part sum mu d, HC part sum beta d}
};

void run_nw_reduce1(const NwJob &j, cudaStream_t st);
// D: the largest distance (the histogram has D + 1 rows).
void run_nw_reduce2(const NwJob &j, int64_t D, cudaStream_t st);

// TS[d * k + i] = sum over d' >= d of d' * hist[d' * k + i], d = 0..D + 1.
void run_nw_tail(const unsigned long long *hist, int64_t D, int k, uint64_t *TS,
                 cudaStream_t st);

struct NwFinal {
    int64_t n, D;
    int k, hybrid;
    uint32_t a, b;
    uint64_t B;                     // sum of all weights
    const uint64_t *tau;            // device, 2
    const int32_t *sidx, *pivot;
    const uint32_t *delta, *beta;
    const unsigned long long *S;
    const uint64_t *wsum, *lc, *TS;
    double *s_hat[2], *clo[2];      // any may be null
};

void run_nw_finalize(const NwFinal &f, cudaStream_t st);

}  // namespace ccg
