// Host launchers of the estimator kernels (estimate.cu).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/cc.h"

namespace ccg {

// LCnum carries this bit when L(v) misses some sampled node (second pass
// needed for LCsum).
constexpr uint64_t kPartialBit = 1ull << 63;

struct HybPrep {
    uint64_t Hsum, Hnum, thr, LCnum;
};

// A level count known on the device (p: the traversal's control block, so
// the host need not wait for it) or on the host (h, when p is null).
struct DevCount {
    const int *p;
    int64_t h;
};

// Error-estimate input flags written by the hybrid preparation (null: the
// error estimate is not wanted).
struct SqPrep {
    uint8_t *flag;
};

struct FinalizeArgs {
    int64_t n;
    int k;
    int hybrid;
    const int32_t *sidx, *pivot;
    const uint32_t *delta;
    const uint64_t *sum2, *S_samp, *lc2;
    const HybPrep *hp;
    double *s_hat[CC_NUM_EST];
    double *clo[CC_NUM_EST];
    uint64_t *hyb_int;
    uint64_t *sample_sum;
    // copies of pivot and delta into the caller's device buffers (else null)
    int32_t *pivot_out;
    uint32_t *delta_out;
    // error estimate (null sq_err: not wanted)
    double *sq_err;
    const uint64_t *hcse;  // n x 2: 128-bit sum of squared errors over HC(v)
    const uint32_t *fdist, *dcc;
    const int32_t *istar;
    // Optional shortcuts, bit-identical to the divisions they replace:
    // inv_k = 1/k when k is a power of two (then x/k = x * inv_k exactly);
    // clo1[2p, 2p+1] = S(c_p), (n-1)/S(c_p); est2t / clo2t[p * tstride + d] =
    // the pivoting upper bound S(c_p) + (n-1) d and its closeness, for
    // d < tstride.
    double inv_k;
    const double *clo1, *est2t, *clo2t;
    int64_t tstride;
    // clo0t[2s, 2s+1] = the sampling estimate and its closeness for sum s,
    // 0 < s < c0len.
    const double *clo0t;
    int64_t c0len;
};

void run_fill_i32(int32_t *p, int64_t n, int32_t v, cudaStream_t st);
void run_scatter_sidx(int32_t *sidx, const int32_t *src, int k, cudaStream_t st);
void run_S_sampled(const uint32_t *hist, DevCount D, int k, const uint32_t *dcc, uint64_t *S,
                   cudaStream_t st);
// TN / TS rows of `stride` >= D + 1 entries.
void run_tail(const uint32_t *hist, DevCount D, int64_t stride, int k, uint64_t *TN,
              uint64_t *TS, cudaStream_t st);
void run_maxdelta(const uint32_t *dcc, int k, uint32_t *maxd, cudaStream_t st);
void run_hyb_prep(int mode, int64_t n, int k, DevCount D, int64_t stride, uint32_t a, uint32_t b,
                  const int32_t *sidx, const int32_t *pivot, const uint32_t *delta,
                  const uint32_t *dcc, const uint32_t *maxd, const uint64_t *TN,
                  const uint64_t *TS, HybPrep *hp, unsigned *npartial, const SqPrep &sq,
                  cudaStream_t st);
void run_istar(const uint32_t *dcc, int k, int32_t *istar, cudaStream_t st);
void run_adaptive_select(int64_t n, int e, const int32_t *sidx, const double *est,
                         const double *sq, double *best_est, double *best_sq, int32_t *choice,
                         cudaStream_t st);
void run_closeness(int64_t n, const double *s_hat, double *clo, cudaStream_t st);
// gate (may be null): skip when gate[0] = gate[1] = 0 (no node needs the
// second pass).
void run_lmask(int64_t n, int W, int k, const int32_t *sidx, const int32_t *pivot,
               const uint32_t *dcc, const HybPrep *hp, uint64_t *Lmask, const unsigned *gate,
               cudaStream_t st);
void run_finalize(const FinalizeArgs &a, cudaStream_t st);
// After a first pass with RED_BAND (rows of rowb bytes) and the hybrid
// preparation: LCsum / LCsumSq into lc2 from the pass's sums over HC(v)
// (hc2) and the deferred bits, and gate[2] of the second pass (zero unless a band
// offset overflowed).
void run_band_resolve(int64_t n, int k, int rowb, const int32_t *sidx, const int32_t *pivot,
                      const uint32_t *delta, const uint32_t *dcc, const HybPrep *hp,
                      const uint8_t *bflag, const uint8_t *band, const uint64_t *sum2,
                      const uint64_t *hc2, uint64_t *lc2, const int *band_ovf, unsigned *gate,
                      const unsigned *npartial, cudaStream_t st);
// Tables of the pivoting estimators for FinalizeArgs (d <= D only).
void run_pivot_tables(int64_t n, int k, const uint64_t *S_samp, DevCount D, int64_t tstride,
                      double *clo1, double *est2t, double *clo2t, double inv_k,
                      int64_t c0len, double *clo0t, cudaStream_t st);

}  // namespace ccg
