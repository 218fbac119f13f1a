// Device functions of the estimator pipeline (estimate.cu): each takes an
// explicit (start, stride) or source index so that the same code runs as a
// stand-alone kernel or inside a team of the batched persistent launch.
#pragma once
#include <cstdint>

#include "cc_internal.h"
#include "estimate.h"

namespace ccg {
namespace {

typedef unsigned __int128 u128;
constexpr int kTailThreads = 256;

// Round-to-nearest-even conversion of an unsigned 128-bit integer: the top
// 64 significant bits with every lower bit folded into a sticky bit are
// converted by the hardware (correctly rounded), then scaled by a power of
// two (exact).
__device__ __forceinline__ double u128_to_double(u128 x)
{
    const uint64_t hi = (uint64_t)(x >> 64);
    if (hi == 0) return (double)(uint64_t)x;
    const int lz = __clzll((long long)hi);
    const u128 y = x << lz;
    uint64_t top = (uint64_t)(y >> 64);
    if ((uint64_t)y != 0) top |= 1ull;
    return ldexp((double)top, 64 - lz);
}

__device__ __forceinline__ void d_fill_i32(int32_t *p, int64_t n, int32_t v, int64_t i0,
                                int64_t stride)
{
    for (int64_t i = i0; i < n;
         i += stride)
        p[i] = v;
}

__device__ __forceinline__ void d_scatter_sidx(int32_t *sidx, const int32_t *src, int k,
                                               int64_t i0, int64_t stride)
{
    for (int64_t i = i0; i < k; i += stride) sidx[src[i]] = (int32_t)i;
}

// S(c_i) = sum over levels l of l * |{v not in C at distance l}| plus the
// distances to the sampled nodes (row i of delta_cc).  A warp per source
// (warp w0 of nw), lanes striding over the levels and the row.
__device__ __forceinline__ void d_S_sampled(const uint32_t *hist, int D, int k,
                                            const uint32_t *dcc, uint64_t *S, int64_t w0,
                                            int64_t nw)
{
    const int lane = threadIdx.x & 31;
    for (int64_t i = w0; i < k; i += nw) {
        unsigned long long s = 0;
        for (int l = 1 + lane; l <= D; l += 32) s += (uint64_t)l * hist[(int64_t)l * k + i];
        for (int j = lane; j < k; j += 32) s += dcc[i * k + j];
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        if (lane == 0) S[i] = s;
    }
}

// Tail tables of the per-source distance histogram: TN[i][t] = number of
// nodes of V \ C farther than t from c_i, TS[i][t] = the sum of their
// distances, t = 0..D (row stride `stride` >= D + 1).  (Role of Algorithm 1's reverse scan of the
// bin/count arrays.)  One CTA per source scans the histogram downwards in
// tiles with a shared-memory suffix scan.
__device__ __forceinline__ void d_tail_source(const uint32_t *hist, int64_t D, int k,
                                              uint64_t *TN, uint64_t *TS, int i,
                                              int64_t stride)
{
    __shared__ unsigned long long sN[kTailThreads], sS[kTailThreads];
    const int tid = threadIdx.x;
    unsigned long long cn = 0, cs = 0;
    for (int64_t top = D; top >= 0; top -= kTailThreads) {
        const int64_t t = top - tid;
        const unsigned long long h = t >= 0 ? hist[t * k + i] : 0ull;
        sN[tid] = h;
        sS[tid] = t >= 0 ? (unsigned long long)t * h : 0ull;
        __syncthreads();
        for (int o = 1; o < kTailThreads; o <<= 1) {
            unsigned long long a = 0, b = 0;
            if (tid >= o) { a = sN[tid - o]; b = sS[tid - o]; }
            __syncthreads();
            sN[tid] += a;
            sS[tid] += b;
            __syncthreads();
        }
        if (t >= 0) {
            TN[(int64_t)i * stride + t] = cn + sN[tid] - h;
            TS[(int64_t)i * stride + t] = cs + sS[tid] - (unsigned long long)t * h;
        }
        cn += sN[kTailThreads - 1];
        cs += sS[kTailThreads - 1];
        __syncthreads();
    }
}

// maxd[p] = largest distance from c_p to a sampled node: a warp per row
// (warp w0 of nw).
__device__ __forceinline__ void d_maxdelta(const uint32_t *dcc, int k, uint32_t *maxd,
                                           int64_t w0, int64_t nw)
{
    const int lane = threadIdx.x & 31;
    for (int64_t p = w0; p < k; p += nw) {
        uint32_t m = 0;
        for (int i = lane; i < k; i += 32) m = max(m, dcc[p * k + i]);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        if (lane == 0) maxd[p] = m;
    }
}

// Per sampled node p: the sampled node farthest from it other than itself
// (ties to the smallest index; p itself when k = 1) -- the stand-in for
// HC(v) in the error estimate of nodes whose HC(v) is empty (section 4).
__device__ __forceinline__ void d_istar(const uint32_t *dcc, int k, int32_t *istar,
                                        int64_t i0, int64_t stride)
{
    for (int64_t p = i0; p < k; p += stride) {
        int best = (int)p;
        for (int i = 0; i < k; ++i)
            if (i != (int)p && (best == (int)p || dcc[p * k + i] > dcc[p * k + best])) best = i;
        istar[p] = best;
    }
}

// Per unsampled node: threshold t = floor(Delta * den / num) (so that "d >
// Delta/eps" is "d > t" for integer d), H statistics from the tail tables of
// the pivot, |L cap C| and whether L(v) misses some sampled node (then the
// hybrid needs the second pass).
// mode & 1: thresholds and |L cap C| (needs delta_cc); mode & 2: H
// statistics from the tail tables (needs the histogram of the pass that
// produced it).  With sq.flag, also which error-estimate input the second
// pass must gather per node: 1 when some c_i is beyond the threshold (the
// squared errors over them), 2 when none is (the distance to the farthest
// sampled node from the pivot) -- with mode 3 only where H(v) is not empty;
// npartial[1] counts the 2s.
__device__ __forceinline__ void d_hyb_prep(int mode, int64_t n, int k, int64_t D,
                           int64_t tstride, uint32_t a, uint32_t b,
                           const int32_t *sidx, const int32_t *pivot,
                           const uint32_t *delta, const uint32_t *dcc,
                           const uint32_t *maxd, const uint64_t *TN, const uint64_t *TS,
                           HybPrep *hp, unsigned *npartial, const SqPrep &sq, int64_t i0,
                                int64_t stride)
{
    for (int64_t v = i0; v < n;
         v += stride) {
        HybPrep h = (mode & 1) ? HybPrep{0, 0, 0, 0} : hp[v];
        if (sidx[v] < 0) {
            const int p = pivot[v];
            const uint64_t t = (uint64_t)delta[v] * b / a;
            if (mode & 2) {
                const int64_t tt = t < (uint64_t)D ? (int64_t)t : D;
                h.Hnum = TN[(int64_t)p * tstride + tt];
                h.Hsum = TS[(int64_t)p * tstride + tt];
            }
            if (mode & 1) {
                h.thr = t;
                if (t >= maxd[p]) {
                    h.LCnum = (uint64_t)k;
                    if (sq.flag) {
                        const uint8_t f = (!(mode & 2) || h.Hnum > 0) ? 2 : 0;
                        sq.flag[v] = f;
                        if (f) atomicAdd(&npartial[1], 1u);
                    }
                } else {
                    uint64_t c = 0;
                    for (int i = 0; i < k; ++i) c += dcc[(int64_t)p * k + i] <= t;
                    h.LCnum = c | kPartialBit;
                    atomicAdd(npartial, 1u);
                    if (sq.flag) sq.flag[v] = 1;
                }
            }
        } else if (sq.flag && (mode & 1)) {
            sq.flag[v] = 0;
        }
        hp[v] = h;
    }
}

// L(v) cap C as a bit mask per (node, word): bit i set when the pivot's
// distance to c_i is at most the threshold.  Zero for sampled nodes.
__device__ __forceinline__ void d_lmask(int64_t n, int W, int k, const int32_t *sidx, const int32_t *pivot,
                        const uint32_t *dcc, const HybPrep *hp, uint64_t *Lmask, int64_t i0,
                                int64_t stride)
{
    for (int64_t i = i0; i < n * W;
         i += stride) {
        const int64_t v = i / W;
        const int w = (int)(i % W);
        uint64_t m = 0;
        // Only nodes whose L(v) misses a sampled node accumulate in the
        // second pass; the others take LCsum = sum.
        if (sidx[v] < 0 && (hp[v].LCnum & kPartialBit)) {
            const int p = pivot[v];
            const uint64_t t = hp[v].thr;
            const int lo = w * 64, hi = min(k, lo + 64);
            for (int s = lo; s < hi; ++s)
                if (dcc[(int64_t)p * k + s] <= t) m |= 1ull << (s - lo);
        }
        Lmask[i] = m;
    }
}

// After a first pass with RED_BAND, for the nodes whose L(v) misses a
// sampled node: hc2 holds the sums over the bits settled in HC(v) on
// arrival (when bflag bit 2 is set); each deferred bit (a lane per source,
// a warp per node: warp w0, w0 + wstride, ...) whose sampled node lies
// beyond the threshold from the pivot joins them with its level l = thr -
// Delta + offset; then LCsum = sum - those and LCsumSq = sumsq - their
// squares, into lc2 (hc2 may be lc2; apart, the first pass's state stays
// intact for another eps-independent use).  Called by whole warps.
__device__ __forceinline__ void d_band_resolve(int64_t n, int k, int rowb, const int32_t *sidx,
                                               const int32_t *pivot, const uint32_t *delta,
                                               const uint32_t *dcc, const HybPrep *hp,
                                               const uint8_t *bflag, const uint8_t *band,
                                               const uint64_t *sum2, const uint64_t *hc2,
                                               uint64_t *lc2, int64_t w0, int64_t wstride)
{
    const int lane = threadIdx.x & 31;
    for (int64_t v = w0; v < n; v += wstride) {
        if (sidx[v] >= 0 || !(hp[v].LCnum & kPartialBit)) continue;
        const uint8_t f = bflag[v];
        uint64_t s = 0, s2 = 0;
        if (f & 1) {
            const int p = pivot[v];
            const uint64_t t = hp[v].thr;
            const uint64_t base = t - delta[v];
            const uint8_t *row = band + v * rowb;  // valid: bflag bit 1
            for (int i = lane; i < k; i += 32) {
                const uint32_t o = row[i];
                if (o && dcc[(int64_t)p * k + i] > t) {
                    const uint64_t l = base + o;
                    s += l;
                    s2 += l * l;
                }
            }
#pragma unroll
            for (int x = 16; x >= 1; x >>= 1) {
                s += __shfl_xor_sync(0xFFFFFFFFu, s, x);
                s2 += __shfl_xor_sync(0xFFFFFFFFu, s2, x);
            }
        }
        if (lane == 0) {
            const uint64_t h1 = (f & 2) ? hc2[2 * v] : 0, h2 = (f & 2) ? hc2[2 * v + 1] : 0;
            lc2[2 * v] = sum2[2 * v] - h1 - s;
            lc2[2 * v + 1] = sum2[2 * v + 1] - h2 - s2;
        }
    }
}

__device__ __forceinline__ void d_finalize(FinalizeArgs A, int64_t i0,
                                int64_t stride)
{
    for (int64_t v = i0; v < A.n;
         v += stride) {
        const uint64_t nm1 = (uint64_t)(A.n - 1);
        const int j = A.sidx[v];
        const uint64_t sum = A.sum2[2 * v];
        double est[CC_NUM_EST], clo[CC_NUM_EST];
        uint64_t h6[6] = {0, 0, 0, 0, 0, 0};
        if (j >= 0) {
            const double ex = (double)A.S_samp[j];
            est[0] = est[1] = est[2] = est[3] = ex;
            clo[0] = clo[1] = clo[2] = clo[3] = (double)nm1 / ex;
        } else {
            const int p = A.pivot[v];
            const uint64_t Sp = A.S_samp[p];
            const bool t0 = A.clo0t && sum > 0 && sum < (uint64_t)A.c0len;
            if (t0) {
                est[0] = A.clo0t[2 * sum];
            } else {
                const double x0 = u128_to_double((u128)nm1 * sum);
                est[0] = A.inv_k != 0.0 ? x0 * A.inv_k : x0 / (double)A.k;
            }
            // closeness of the sampling estimate, also reused by the hybrid
            auto clo_sampling = [&]() {
                return t0 ? A.clo0t[2 * sum + 1] : (double)nm1 / est[0];
            };
            clo[0] = A.clo[0] ? clo_sampling() : 0.0;
            est[1] = A.clo1 ? A.clo1[2 * p] : (double)Sp;
            clo[1] = A.clo1 ? A.clo1[2 * p + 1] : (A.clo[1] ? (double)nm1 / est[1] : 0.0);
            const uint32_t d = A.delta[v];
            if (A.est2t && d < A.tstride) {
                est[2] = A.est2t[(int64_t)p * A.tstride + d];
                clo[2] = A.clo2t[(int64_t)p * A.tstride + d];
            } else {
                est[2] = u128_to_double((u128)Sp + (u128)nm1 * d);
                clo[2] = A.clo[2] ? (double)nm1 / est[2] : 0.0;
            }
            est[3] = 0.0;
            clo[3] = 0.0;
            if (A.hybrid) {
                const HybPrep h = A.hp[v];
                const uint64_t LCnum = h.LCnum & ~kPartialBit;
                const bool partial = (h.LCnum & kPartialBit) != 0;
                const uint64_t LCsum = partial ? A.lc2[2 * v] : sum;
                const uint64_t LCsq = partial ? A.lc2[2 * v + 1] : A.sum2[2 * v + 1];
                const uint64_t HCsum = sum - LCsum;
                const uint64_t HCnum = (uint64_t)A.k - LCnum;
                const uint64_t Lnum = nm1 - h.Hnum - HCnum;
                const u128 N = (u128)(h.Hsum + HCsum) * LCnum + (u128)LCsum * Lnum;
                if (LCnum == (uint64_t)A.k && h.Hnum == 0) {
                    // N = sum * (n-1): the sampling estimate, bit for bit.
                    est[3] = est[0];
                    clo[3] = A.clo[3] ? (A.clo[0] ? clo[0] : clo_sampling()) : 0.0;
                } else {
                    const double xN = u128_to_double(N);
                    est[3] = (LCnum == (uint64_t)A.k && A.inv_k != 0.0) ? xN * A.inv_k
                                                                         : xN / (double)LCnum;
                    clo[3] = A.clo[3] ? (double)nm1 / est[3] : 0.0;
                }
                h6[0] = h.Hsum; h6[1] = h.Hnum; h6[2] = HCsum;
                h6[3] = LCsum; h6[4] = LCnum; h6[5] = LCsq;
                if (A.sq_err) {
                    // SqErrEst (Algorithm 1's last loop; section 4): the
                    // sampling term |L| var(L n C) / |L n C| and the pivoting
                    // term |H| * mean over HC of (d(c_i, v) - d(c(v), c_i))^2.
                    const u128 var_num = (u128)LCsq * LCnum - (u128)LCsum * LCsum;
                    const double t1 = u128_to_double(var_num * Lnum) /
                                      ((double)LCnum * (double)LCnum * (double)LCnum);
                    double t2 = 0.0;
                    if (HCnum > 0) {
                        const u128 e2 = ((u128)A.hcse[2 * v + 1] << 64) | A.hcse[2 * v];
                        t2 = u128_to_double(e2 * h.Hnum) / (double)HCnum;
                    } else if (h.Hnum > 0) {
                        const int is = A.istar[p];
                        const int64_t e = (int64_t)A.fdist[v] -
                                          (int64_t)A.dcc[(int64_t)p * A.k + is];
                        const uint64_t ae = (uint64_t)(e < 0 ? -e : e);
                        t2 = u128_to_double((u128)ae * ae * h.Hnum);
                    }
                    A.sq_err[v] = t1 + t2;
                }
            }
        }
        if (j >= 0 && A.sq_err) A.sq_err[v] = 0.0;
        for (int e = 0; e < CC_NUM_EST; ++e) {
            if (e == CC_EST_HYBRID && !A.hybrid) continue;
            if (A.s_hat[e]) A.s_hat[e][v] = est[e];
            if (A.clo[e]) A.clo[e][v] = clo[e];
        }
        if (A.hyb_int && A.hybrid)
            for (int q = 0; q < 6; ++q) A.hyb_int[6 * v + q] = h6[q];
        if (A.sample_sum) A.sample_sum[v] = sum;
        if (A.pivot_out) A.pivot_out[v] = A.pivot[v];
        if (A.delta_out) A.delta_out[v] = A.delta[v];
    }
}

}  // namespace
}  // namespace ccg
