// Per-source and per-node kernels around the traversal passes: exact S of
// the sampled nodes, the H tail tables, the hybrid thresholds and L(v)
// masks, and the FP64 finalisation of the four estimators (section 2,
// eqs. (3) and (4); Algorithm 1's final loop).
#include <cstdint>

#include "estimate_dev.cuh"

namespace ccg {

namespace {

#define GSTART (blockIdx.x * (int64_t)blockDim.x + threadIdx.x)
#define GSTRIDE ((int64_t)gridDim.x * blockDim.x)

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v)
{
    d_fill_i32(p, n, v, GSTART, GSTRIDE);
}

__global__ void k_scatter_sidx(int32_t *sidx, const int32_t *src, int k)
{
    d_scatter_sidx(sidx, src, k, GSTART, GSTRIDE);
}

__device__ __forceinline__ int64_t count_of(DevCount c) { return c.p ? (int64_t)*c.p : c.h; }

__global__ void k_S_sampled(const uint32_t *hist, DevCount D, int k, const uint32_t *dcc,
                            uint64_t *S)
{
    d_S_sampled(hist, (int)count_of(D), k, dcc, S, GSTART >> 5, GSTRIDE >> 5);
}

__global__ void k_tail(const uint32_t *hist, DevCount D, int64_t stride, int k, uint64_t *TN,
                       uint64_t *TS)
{
    d_tail_source(hist, count_of(D), k, TN, TS, blockIdx.x, stride);
}

__global__ void k_maxdelta(const uint32_t *dcc, int k, uint32_t *maxd)
{
    d_maxdelta(dcc, k, maxd, GSTART >> 5, GSTRIDE >> 5);
}

__global__ void k_hyb_prep(int mode, int64_t n, int k, DevCount D, int64_t stride, uint32_t a,
                           uint32_t b, const int32_t *sidx, const int32_t *pivot,
                           const uint32_t *delta, const uint32_t *dcc,
                           const uint32_t *maxd, const uint64_t *TN, const uint64_t *TS,
                           HybPrep *hp, unsigned *npartial, SqPrep sq)
{
    d_hyb_prep(mode, n, k, count_of(D), stride, a, b, sidx, pivot, delta, dcc, maxd, TN, TS,
               hp, npartial, sq, GSTART, GSTRIDE);
}

__global__ void k_istar(const uint32_t *dcc, int k, int32_t *istar)
{
    d_istar(dcc, k, istar, GSTART, GSTRIDE);
}

__global__ void k_lmask(int64_t n, int W, int k, const int32_t *sidx, const int32_t *pivot,
                        const uint32_t *dcc, const HybPrep *hp, uint64_t *Lmask,
                        const unsigned *gate)
{
    if (gate && gate[0] == 0u && gate[1] == 0u) return;
    d_lmask(n, W, k, sidx, pivot, dcc, hp, Lmask, GSTART, GSTRIDE);
}

__global__ void k_finalize(FinalizeArgs A)
{
    d_finalize(A, GSTART, GSTRIDE);
}

// After a first pass with RED_BAND: the gate of the second pass (it runs
// only when a band offset overflowed and some node needs it), then LCsum /
// LCsumSq of the nodes whose L(v) misses a sampled node (d_band_resolve);
// nothing more when no node does.
__global__ void k_band_resolve(int64_t n, int k, int rowb, const int32_t *sidx,
                               const int32_t *pivot, const uint32_t *delta, const uint32_t *dcc,
                               const HybPrep *hp, const uint8_t *bflag, const uint8_t *band,
                               const uint64_t *sum2, const uint64_t *hc2, uint64_t *lc2,
                               const int *band_ovf, const unsigned *npartial, unsigned *gate)
{
    const bool ovf = *band_ovf != 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        gate[0] = ovf ? npartial[0] + npartial[1] : 0u;
        gate[1] = 0u;
    }
    if (ovf || npartial[0] == 0) return;  // the second pass, or nothing, to do
    d_band_resolve(n, k, rowb, sidx, pivot, delta, dcc, hp, bflag, band, sum2, hc2, lc2,
                   (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5,
                   ((int64_t)gridDim.x * blockDim.x) >> 5);
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

void run_S_sampled(const uint32_t *hist, DevCount D, int k, const uint32_t *dcc, uint64_t *S,
                   cudaStream_t st)
{
    k_S_sampled<<<(k + 7) / 8, 256, 0, st>>>(hist, D, k, dcc, S);
}

void run_tail(const uint32_t *hist, DevCount D, int64_t stride, int k, uint64_t *TN,
              uint64_t *TS, cudaStream_t st)
{
    k_tail<<<k, kTailThreads, 0, st>>>(hist, D, stride, k, TN, TS);
}

void run_maxdelta(const uint32_t *dcc, int k, uint32_t *maxd, cudaStream_t st)
{
    k_maxdelta<<<(k + 7) / 8, 256, 0, st>>>(dcc, k, maxd);
}

void run_hyb_prep(int mode, int64_t n, int k, DevCount D, int64_t stride, uint32_t a,
                  uint32_t b, const int32_t *sidx, const int32_t *pivot, const uint32_t *delta,
                  const uint32_t *dcc, const uint32_t *maxd, const uint64_t *TN,
                  const uint64_t *TS, HybPrep *hp, unsigned *npartial, const SqPrep &sq,
                  cudaStream_t st)
{
    k_hyb_prep<<<grid_for(n, 256), 256, 0, st>>>(mode, n, k, D, stride, a, b, sidx, pivot,
                                                 delta, dcc, maxd, TN, TS, hp, npartial, sq);
}

// Adaptive hybrid (section 6): keep, per node, the estimate of the eps with
// the smallest error estimate so far (entry e of the list; ties keep the
// earlier one); sampled nodes keep their exact S, error 0 and choice -1.
__global__ void k_adaptive_select(int64_t n, int e, const int32_t *sidx, const double *est,
                                  const double *sq, double *best_est, double *best_sq,
                                  int32_t *choice)
{
    for (int64_t v = GSTART; v < n; v += GSTRIDE) {
        if (sidx[v] >= 0) {
            best_est[v] = est[v];
            best_sq[v] = 0.0;
            choice[v] = -1;
        } else if (e == 0 || sq[v] < best_sq[v]) {
            best_est[v] = est[v];
            best_sq[v] = sq[v];
            choice[v] = e;
        }
    }
}

__global__ void k_closeness(int64_t n, const double *s_hat, double *clo)
{
    for (int64_t v = GSTART; v < n; v += GSTRIDE) clo[v] = (double)(n - 1) / s_hat[v];
}

void run_adaptive_select(int64_t n, int e, const int32_t *sidx, const double *est,
                         const double *sq, double *best_est, double *best_sq, int32_t *choice,
                         cudaStream_t st)
{
    k_adaptive_select<<<grid_for(n, 256), 256, 0, st>>>(n, e, sidx, est, sq, best_est, best_sq,
                                                        choice);
}

// clo1[2p, 2p+1] = S(c_p) and (n-1)/S(c_p); est2t / clo2t[p * tstride + d]
// = S(c_p) + (n-1) d and its closeness, for d <= D (the pivoting estimators
// take only these values); clo0t[2s, 2s+1] = the sampling estimate and its
// closeness for sum s (0 < s < c0len, s <= k D), computed exactly as the
// finalisation would.  The pairs make a finalisation of a graph of small
// diameter table lookups only (FP64 is slow on this part).
__global__ void k_pivot_tables(int64_t n, int k, const uint64_t *S_samp, DevCount D,
                               int64_t tstride, double *clo1, double *est2t, double *clo2t,
                               double inv_k, int64_t c0len, double *clo0t)
{
    const int64_t Dv = count_of(D);
    const uint64_t nm1 = (uint64_t)(n - 1);
    const int64_t smax = min(c0len, (int64_t)k * Dv + 1);
    for (int64_t s = GSTART + 1; s < smax; s += GSTRIDE) {
        const double x0 = u128_to_double((u128)nm1 * (uint64_t)s);
        const double e0 = inv_k != 0.0 ? x0 * inv_k : x0 / (double)k;
        clo0t[2 * s] = e0;
        clo0t[2 * s + 1] = (double)nm1 / e0;
    }
    const int64_t dn = min(tstride, Dv + 1);  // distances 0 .. dn-1 per pivot
    for (int64_t q = GSTART; q < (int64_t)k * dn; q += GSTRIDE) {
        const int64_t p = q / dn, d = q % dn;
        const int64_t i = p * tstride + d;
        const uint64_t Sp = S_samp[p];
        const double e2 = u128_to_double((u128)Sp + (u128)nm1 * (uint64_t)d);
        est2t[i] = e2;
        clo2t[i] = (double)nm1 / e2;
        if (d == 0) {
            clo1[2 * p] = (double)Sp;
            clo1[2 * p + 1] = (double)nm1 / (double)Sp;
        }
    }
}

void run_pivot_tables(int64_t n, int k, const uint64_t *S_samp, DevCount D, int64_t tstride,
                      double *clo1, double *est2t, double *clo2t, double inv_k,
                      int64_t c0len, double *clo0t, cudaStream_t st)
{
    // The ranges depend on the level count, read on the device: a fixed
    // grid strides over them.
    k_pivot_tables<<<152 * 2, 256, 0, st>>>(n, k, S_samp, D, tstride, clo1, est2t, clo2t,
                                            inv_k, c0len, clo0t);
}

void run_closeness(int64_t n, const double *s_hat, double *clo, cudaStream_t st)
{
    k_closeness<<<grid_for(n, 256), 256, 0, st>>>(n, s_hat, clo);
}

void run_istar(const uint32_t *dcc, int k, int32_t *istar, cudaStream_t st)
{
    k_istar<<<(k + 127) / 128, 128, 0, st>>>(dcc, k, istar);
}

void run_lmask(int64_t n, int W, int k, const int32_t *sidx, const int32_t *pivot,
               const uint32_t *dcc, const HybPrep *hp, uint64_t *Lmask, const unsigned *gate,
               cudaStream_t st)
{
    k_lmask<<<grid_for(n * W, 256), 256, 0, st>>>(n, W, k, sidx, pivot, dcc, hp, Lmask, gate);
}

void run_band_resolve(int64_t n, int k, int rowb, const int32_t *sidx, const int32_t *pivot,
                      const uint32_t *delta, const uint32_t *dcc, const HybPrep *hp,
                      const uint8_t *bflag, const uint8_t *band, const uint64_t *sum2,
                      const uint64_t *hc2, uint64_t *lc2, const int *band_ovf, unsigned *gate,
                      const unsigned *npartial, cudaStream_t st)
{
    k_band_resolve<<<grid_for(n * 32, 256), 256, 0, st>>>(n, k, rowb, sidx, pivot, delta, dcc,
                                                          hp, bflag, band, sum2, hc2, lc2,
                                                          band_ovf, npartial, gate);
}

void run_finalize(const FinalizeArgs &a, cudaStream_t st)
{
    k_finalize<<<grid_for(a.n, 256), 256, 0, st>>>(a);
}

}  // namespace ccg
