// Per-source and per-node kernels around the traversal passes: exact S of
// the sampled nodes, the H tail tables, the hybrid thresholds and L(v)
// masks, and the FP64 finalisation of the four estimators (section 2,
// eqs. (3) and (4); Algorithm 1's final loop).
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

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void k_scatter_sidx(int32_t *sidx, const int32_t *src, int k)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) sidx[src[i]] = i;
}

// S(c_i) = sum over levels l of l * |{v not in C at distance l}| plus the
// distances to the sampled nodes (row i of delta_cc).
__global__ void k_S_sampled(const uint32_t *hist, int D, int k, const uint32_t *dcc,
                            uint64_t *S)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    uint64_t s = 0;
    for (int l = 1; l <= D; ++l) s += (uint64_t)l * hist[(int64_t)l * k + i];
    for (int j = 0; j < k; ++j) s += dcc[(int64_t)i * k + j];
    S[i] = s;
}

// Tail tables of the per-source distance histogram: TN[i][t] = number of
// nodes of V \ C farther than t from c_i, TS[i][t] = the sum of their
// distances, t = 0..D.  (Role of Algorithm 1's reverse scan of the
// bin/count arrays.)  One CTA per source scans the histogram downwards in
// tiles with a shared-memory suffix scan.
__global__ void k_tail(const uint32_t *hist, int64_t D, int k, uint64_t *TN, uint64_t *TS)
{
    __shared__ unsigned long long sN[kTailThreads], sS[kTailThreads];
    const int i = blockIdx.x;
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
            TN[(int64_t)i * (D + 1) + t] = cn + sN[tid] - h;
            TS[(int64_t)i * (D + 1) + t] = cs + sS[tid] - (unsigned long long)t * h;
        }
        cn += sN[kTailThreads - 1];
        cs += sS[kTailThreads - 1];
        __syncthreads();
    }
}

__global__ void k_maxdelta(const uint32_t *dcc, int k, uint32_t *maxd)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= k) return;
    uint32_t m = 0;
    for (int i = 0; i < k; ++i) m = max(m, dcc[(int64_t)p * k + i]);
    maxd[p] = m;
}

// Per unsampled node: threshold t = floor(Delta * den / num) (so that "d >
// Delta/eps" is "d > t" for integer d), H statistics from the tail tables of
// the pivot, |L cap C| and whether L(v) misses some sampled node (then the
// hybrid needs the second pass).
// mode & 1: thresholds and |L cap C| (needs delta_cc); mode & 2: H
// statistics from the tail tables (needs the histogram of the pass that
// produced it).
__global__ void k_hyb_prep(int mode, int64_t n, int k, int64_t D, uint32_t a, uint32_t b,
                           const int32_t *sidx, const int32_t *pivot,
                           const uint32_t *delta, const uint32_t *dcc,
                           const uint32_t *maxd, const uint64_t *TN, const uint64_t *TS,
                           HybPrep *hp, unsigned *npartial)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        HybPrep h = (mode & 1) ? HybPrep{0, 0, 0, 0} : hp[v];
        if (sidx[v] < 0) {
            const int p = pivot[v];
            const uint64_t t = (uint64_t)delta[v] * b / a;
            if (mode & 2) {
                const int64_t tt = t < (uint64_t)D ? (int64_t)t : D;
                h.Hnum = TN[(int64_t)p * (D + 1) + tt];
                h.Hsum = TS[(int64_t)p * (D + 1) + tt];
            }
            if (mode & 1) {
                h.thr = t;
                if (t >= maxd[p]) {
                    h.LCnum = (uint64_t)k;
                } else {
                    uint64_t c = 0;
                    for (int i = 0; i < k; ++i) c += dcc[(int64_t)p * k + i] <= t;
                    h.LCnum = c | kPartialBit;
                    atomicAdd(npartial, 1u);
                }
            }
        }
        hp[v] = h;
    }
}

// L(v) cap C as a bit mask per (node, word): bit i set when the pivot's
// distance to c_i is at most the threshold.  Zero for sampled nodes.
__global__ void k_lmask(int64_t n, int W, int k, const int32_t *sidx, const int32_t *pivot,
                        const uint32_t *dcc, const HybPrep *hp, uint64_t *Lmask)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * W;
         i += (int64_t)gridDim.x * blockDim.x) {
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

__global__ void k_finalize(FinalizeArgs A)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < A.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t nm1 = (uint64_t)(A.n - 1);
        const int j = A.sidx[v];
        const uint64_t sum = A.sum2[2 * v];
        double est[CC_NUM_EST];
        uint64_t h6[6] = {0, 0, 0, 0, 0, 0};
        if (j >= 0) {
            const double ex = (double)A.S_samp[j];
            est[0] = est[1] = est[2] = est[3] = ex;
        } else {
            const int p = A.pivot[v];
            const uint64_t Sp = A.S_samp[p];
            est[0] = u128_to_double((u128)nm1 * sum) / (double)A.k;
            est[1] = (double)Sp;
            est[2] = u128_to_double((u128)Sp + (u128)nm1 * A.delta[v]);
            est[3] = 0.0;
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
                est[3] = u128_to_double(N) / (double)LCnum;
                h6[0] = h.Hsum; h6[1] = h.Hnum; h6[2] = HCsum;
                h6[3] = LCsum; h6[4] = LCnum; h6[5] = LCsq;
            }
        }
        for (int e = 0; e < CC_NUM_EST; ++e) {
            if (e == CC_EST_HYBRID && !A.hybrid) continue;
            if (A.s_hat[e]) A.s_hat[e][v] = est[e];
            if (A.clo[e]) A.clo[e][v] = (double)nm1 / est[e];
        }
        if (A.hyb_int && A.hybrid)
            for (int q = 0; q < 6; ++q) A.hyb_int[6 * v + q] = h6[q];
        if (A.sample_sum) A.sample_sum[v] = sum;
    }
}

inline int grid_for(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    if (g > 152 * 32) g = 152 * 32;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

void run_fill_i32(int32_t *p, int64_t n, int32_t v, cudaStream_t st)
{
    k_fill_i32<<<grid_for(n, 256), 256, 0, st>>>(p, n, v);
}

void run_scatter_sidx(int32_t *sidx, const int32_t *src, int k, cudaStream_t st)
{
    k_scatter_sidx<<<(k + 255) / 256, 256, 0, st>>>(sidx, src, k);
}

void run_S_sampled(const uint32_t *hist, int D, int k, const uint32_t *dcc, uint64_t *S,
                   cudaStream_t st)
{
    k_S_sampled<<<(k + 127) / 128, 128, 0, st>>>(hist, D, k, dcc, S);
}

void run_tail(const uint32_t *hist, int64_t D, int k, uint64_t *TN, uint64_t *TS,
              cudaStream_t st)
{
    k_tail<<<k, kTailThreads, 0, st>>>(hist, D, k, TN, TS);
}

void run_maxdelta(const uint32_t *dcc, int k, uint32_t *maxd, cudaStream_t st)
{
    k_maxdelta<<<(k + 127) / 128, 128, 0, st>>>(dcc, k, maxd);
}

void run_hyb_prep(int mode, int64_t n, int k, int64_t D, uint32_t a, uint32_t b,
                  const int32_t *sidx, const int32_t *pivot, const uint32_t *delta,
                  const uint32_t *dcc, const uint32_t *maxd, const uint64_t *TN,
                  const uint64_t *TS, HybPrep *hp, unsigned *npartial, cudaStream_t st)
{
    k_hyb_prep<<<grid_for(n, 256), 256, 0, st>>>(mode, n, k, D, a, b, sidx, pivot, delta,
                                                 dcc, maxd, TN, TS, hp, npartial);
}

void run_lmask(int64_t n, int W, int k, const int32_t *sidx, const int32_t *pivot,
               const uint32_t *dcc, const HybPrep *hp, uint64_t *Lmask, cudaStream_t st)
{
    k_lmask<<<grid_for(n * W, 256), 256, 0, st>>>(n, W, k, sidx, pivot, dcc, hp, Lmask);
}

void run_finalize(const FinalizeArgs &a, cudaStream_t st)
{
    k_finalize<<<grid_for(a.n, 256), 256, 0, st>>>(a);
}

}  // namespace ccg
