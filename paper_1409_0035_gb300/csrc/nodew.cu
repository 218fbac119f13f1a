// Node-weighted closeness (section 5, "Weighted Centrality", and its
// modification of Algorithm 1) on the device.
//
// Sampler: the threshold tau solves sum over v of min(1, beta(v)/tau) = k.
// With the weights sorted b_0 >= b_1 >= ..., the h largest are certain and
// tau = (b_h + b_{h+1} + ...) / (k - h) for the smallest h with
// b_h (k - h) < b_h + b_{h+1} + ... (one sort, one scan, one test per h).
// The draw is systematic sampling with unequal probabilities (Madow 1949)
// along the splitmix64 order of the nodes: an uncertain node occupies an
// interval of beta(v) td on a line of length td tn and the td points
// u, u + tn, ... pick the nodes whose interval holds one, so every node is
// in the sample with probability exactly min(1, beta(v)/tau) and the sample
// has exactly k nodes.  Section 5 draws with VarOpt stream sampling, which
// has the same inclusion probabilities and size; a device holding all the
// weights has no stream to serve.
//
// Estimates: over the chunks of shortest-path rows of the unweighted and
// weighted paths, per node the sum of max(tau, beta(c_i)) d(c_i, v) (times
// td, an integer) and per sampled node the exact S_beta; for the hybrid a
// second sweep splits the sampled nodes into HC (beyond the node's
// threshold from its pivot: weight beta) and the rest (weight max(tau,
// beta)) and builds the beta mass of V \ C per distance from each sampled
// node, whose suffix sums give the H tail.
#include <algorithm>
#include <cstdint>

#include "estimate_dev.cuh"
#include "graph_gpu.h"
#include "nodew.h"

namespace ccg {

namespace {

constexpr int kT = 256;

int grid_for(int64_t n)
{
    return (int)std::min<int64_t>(std::max<int64_t>(1, (n + kT - 1) / kT), 152 * 16);
}

// ---- threshold -----------------------------------------------------------

__global__ void k_total(const uint32_t *beta, int64_t n, unsigned long long *sum)
{
    uint64_t s = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        s += beta[v];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(sum, (unsigned long long)s);
}

__global__ void k_desc_keys(const uint32_t *beta, int64_t n, uint64_t *keys, uint32_t *vals)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        keys[v] = 0xFFFFFFFFull - beta[v];  // ascending keys = descending weights
        vals[v] = (uint32_t)v;
    }
}

__global__ void k_key_to_weight(const uint64_t *keys, int64_t n, uint64_t *b)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        b[j] = 0xFFFFFFFFull - keys[j];
}

// b: weights in descending order; pre: exclusive prefix sums; total: B.
// tau4[2] = number of positive weights; tau4[3] = smallest h with
// b_h (k - h) < B - pre_h (k when none).
__global__ void k_tau_test(const uint64_t *b, const uint64_t *pre, int64_t n, int k,
                           uint64_t total, unsigned long long *tau4)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        if (b[j] > 0 && (j + 1 == n || b[j + 1] == 0)) tau4[2] = (unsigned long long)(j + 1);
        if (j < k && b[j] * (uint64_t)(k - j) < total - pre[j])
            atomicMin(&tau4[3], (unsigned long long)j);
    }
}

__global__ void k_tau_final(const uint64_t *b, const uint64_t *pre, int k, uint64_t total,
                            uint64_t *tau4)
{
    const uint64_t npos = tau4[2];
    if (npos < (uint64_t)k) {
        tau4[0] = tau4[1] = 0;
    } else if (npos == (uint64_t)k) {  // every positive weight certain
        tau4[0] = b[k - 1];
        tau4[1] = 1;
    } else if (tau4[3] < (uint64_t)k) {  // always, with more than k positive weights
        const uint64_t h = tau4[3];
        tau4[0] = total - pre[h];
        tau4[1] = (uint64_t)k - h;
    } else {
        tau4[0] = tau4[1] = 0;
    }
}

// ---- systematic draw -----------------------------------------------------

__global__ void k_order_keys(int64_t n, uint64_t seed, uint64_t *keys, uint32_t *vals)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        keys[v] = splitmix64_out(seed, (uint64_t)v);
        vals[v] = (uint32_t)v;
    }
}

__device__ __forceinline__ bool uncertain(uint64_t b, uint64_t tn, uint64_t td)
{
    return b > 0 && b * td < tn;
}

// Interval length of each node along the order (uncertain nodes only).
__global__ void k_lengths(const uint32_t *order, const uint32_t *beta, const uint64_t *tau,
                          int64_t n, uint64_t *len)
{
    const uint64_t tn = tau[0], td = tau[1];
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t b = beta[order[j]];
        len[j] = uncertain(b, tn, td) ? b * td : 0;
    }
}

// Points u + t tn (t >= 0) below x.
__device__ __forceinline__ uint64_t points_below(uint64_t x, uint64_t u, uint64_t tn)
{
    return x <= u ? 0 : (x - u + tn - 1) / tn;
}

__global__ void k_pick(const uint32_t *order, const uint32_t *beta, const uint64_t *tau,
                       const uint64_t *start, int64_t n, uint64_t seed, uint64_t *flags)
{
    const uint64_t tn = tau[0], td = tau[1];
    const uint64_t u = __umul64hi(splitmix64_out(seed, (uint64_t)n), tn);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t b = beta[order[j]];
        uint64_t f = 0;
        if (b > 0) {
            if (!uncertain(b, tn, td)) {
                f = 1;
            } else {
                const uint64_t lo = start[j], hi = lo + b * td;
                f = points_below(hi, u, tn) > points_below(lo, u, tn) ? 1 : 0;
            }
        }
        flags[j] = f;
    }
}

// out holds k entries; the host checks that exactly k were picked.
__global__ void k_gather_picked(const uint32_t *order, const uint64_t *flags,
                                const uint64_t *pos, int64_t n, int k, int32_t *out)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        if (flags[j] && pos[j] < (uint64_t)k) out[pos[j]] = (int32_t)order[j];
}

// ---- estimates -----------------------------------------------------------

__global__ void k_mu(int k, const int32_t *sources, const uint32_t *beta, const uint64_t *tau,
                     uint32_t *bsrc, uint64_t *mu, unsigned long long *msum)
{
    const uint64_t tn = tau[0], td = tau[1];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const uint64_t b = beta[sources[i]];
        const uint64_t m = b * td >= tn ? b * td : tn;  // max(tau, beta) * td
        bsrc[i] = (uint32_t)b;
        mu[i] = m;
        atomicAdd(&msum[0], (unsigned long long)m);
        if (b == 0) msum[1] = 1;
    }
}

__device__ __forceinline__ uint64_t dist_at(const NwJob &J, int64_t v, int j)
{
    const size_t r = J.row_of ? (size_t)J.row_of[v] : (size_t)v;
    const size_t at = r * J.ld + J.sub + j;
    uint64_t d = J.distF[at];
    if (J.distR) d += J.distR[at];
    return d;
}

__device__ __forceinline__ uint64_t warp_sum64(uint64_t x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    return x;
}

// Both sweeps take kTile nodes per warp at a time with lane = sampled node
// of the slice: the rows of all kTile nodes are loaded first (coalesced, one
// memory round trip per tile), per-source sums stay in the lanes'
// registers, per-node sums are warp-reduced and land on lane u for node u,
// whose read-modify-writes the first kTile lanes then issue together.
constexpr int kTile = 8;

// First sweep: wsum[v] += sum over the slice of mu_i d(c_i, v) and S[i] +=
// sum over v of beta(v) d(c_i, v).
__global__ void __launch_bounds__(kT) k_nw_reduce1(NwJob J)
{
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool valid = lane < J.kc;
    const uint64_t mu = valid ? J.mu[J.base + lane] : 0;
    uint64_t Sacc = 0;
    for (int64_t v0 = gwarp * kTile; v0 < J.n; v0 += nwarps * kTile) {
        uint64_t d[kTile];
#pragma unroll
        for (int u = 0; u < kTile; ++u) d[u] = valid && v0 + u < J.n ? dist_at(J, v0 + u, lane) : 0;
        const uint64_t bl = lane < kTile && v0 + lane < J.n ? J.beta[v0 + lane] : 0;
        uint64_t mine = 0;
#pragma unroll
        for (int u = 0; u < kTile; ++u) {
            if (v0 + u >= J.n) break;  // warp-uniform
            Sacc += __shfl_sync(0xFFFFFFFFu, bl, u) * d[u];
            const uint64_t x = warp_sum64(mu * d[u]);
            if (lane == u) mine = x;
        }
        if (lane < kTile && v0 + lane < J.n) J.wsum[v0 + lane] += mine;
    }
    // one global atomic per (CTA, source): the warps' sums meet in shared
    // memory first
    __shared__ uint64_t s_S[kT / 32][32];
    s_S[threadIdx.x >> 5][lane] = Sacc;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint64_t t = 0;
        for (int w = 0; w < kT / 32; ++w) t += s_S[w][threadIdx.x];
        if (threadIdx.x < J.kc && t)
            atomicAdd(&J.S[J.base + threadIdx.x], (unsigned long long)t);
    }
}

// Second sweep (non-sampled nodes): the HC / L split of the slice's sampled
// nodes and the beta mass per distance from each of them.  With small
// distances (D < kSmemRows) the slice's histogram (D + 1 rows of 32
// columns) is accumulated per CTA in shared memory and added to the global
// one at the end: most nodes share a handful of (distance, source) cells,
// which global atomics would serialise in L2.  A warp's lanes always hit
// different columns.
constexpr int kSmemRows = 192;

__global__ void __launch_bounds__(kT) k_nw_reduce2(NwJob J, int64_t D)
{
    extern __shared__ unsigned long long sh[];
    const bool local = D < kSmemRows;
    const int cells = local ? (int)(D + 1) * 32 : 0;
    for (int c = threadIdx.x; c < cells; c += blockDim.x) sh[c] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool valid = lane < J.kc;
    const int i = J.base + lane;
    const uint64_t mu = valid ? J.mu[i] : 0;
    const uint64_t bs = valid ? J.bsrc[i] : 0;
    for (int64_t v0 = gwarp * kTile; v0 < J.n; v0 += nwarps * kTile) {
        // per-node data on lanes 0..kTile-1
        int32_t sx = 0, pv = 0;
        uint32_t dl = 0, bv = 0;
        if (lane < kTile && v0 + lane < J.n) {
            const int64_t v = v0 + lane;
            sx = J.sidx[v];
            pv = J.pivot[v];
            dl = J.delta[v];
            bv = J.beta[v];
        }
        uint64_t d[kTile];
        uint32_t dc[kTile];
#pragma unroll
        for (int u = 0; u < kTile; ++u) {
            const int32_t p = __shfl_sync(0xFFFFFFFFu, pv, u);
            const bool on = valid && v0 + u < J.n;
            d[u] = on ? dist_at(J, v0 + u, lane) : 0;
            dc[u] = on ? J.dcc[(size_t)p * J.k + i] : 0;
        }
        uint64_t my_l = 0, my_h = 0;
#pragma unroll
        for (int u = 0; u < kTile; ++u) {
            if (v0 + u >= J.n) break;                         // warp-uniform
            if (__shfl_sync(0xFFFFFFFFu, sx, u) >= 0) continue;  // sampled: exact
            const uint64_t thr = (uint64_t)__shfl_sync(0xFFFFFFFFu, dl, u) * J.b;
            const uint32_t b_u = __shfl_sync(0xFFFFFFFFu, bv, u);
            uint64_t lp = 0, hc = 0;
            if (valid) {
                const uint64_t dd = d[u];
                if (b_u) {
                    if (local)
                        atomicAdd(&sh[dd * 32 + lane], (unsigned long long)b_u);
                    else
                        atomicAdd(&J.hist[dd * J.k + i], (unsigned long long)b_u);
                }
                if ((uint64_t)dc[u] * J.a > thr)
                    hc = bs * dd;
                else
                    lp = mu * dd;
            }
            lp = warp_sum64(lp);
            hc = warp_sum64(hc);
            if (lane == u) {
                my_l = lp;
                my_h = hc;
            }
        }
        if (lane < kTile && v0 + lane < J.n && sx < 0) {
            const int64_t v = v0 + lane;
            J.lc[2 * v] += my_l;
            J.lc[2 * v + 1] += my_h;
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < cells; c += blockDim.x) {
        const int j = c & 31;
        if (sh[c] && j < J.kc) atomicAdd(&J.hist[(int64_t)(c >> 5) * J.k + J.base + j], sh[c]);
    }
}

// Suffix sums of d * hist over d for one sampled node per CTA: each thread
// takes a contiguous segment, the segment sums are suffix-scanned in shared
// memory, then every thread writes its segment from the top down.
__global__ void __launch_bounds__(kT) k_nw_tail(const unsigned long long *hist, int64_t D,
                                               int k, uint64_t *TS)
{
    __shared__ uint64_t part[kT];
    const int i = blockIdx.x;
    const int t = threadIdx.x;
    const int64_t rows = D + 2;  // d = 0..D, and D + 1 (empty tail)
    const int64_t seg = (rows + kT - 1) / kT;
    const int64_t lo = t * seg < rows ? t * seg : rows;
    const int64_t hi = lo + seg < rows ? lo + seg : rows;
    uint64_t s = 0;
    for (int64_t d = lo; d < hi && d <= D; ++d) s += (uint64_t)d * hist[d * k + i];
    part[t] = s;
    __syncthreads();
    // inclusive suffix scan over threads
    for (int o = 1; o < kT; o <<= 1) {
        const uint64_t add = t + o < kT ? part[t + o] : 0;
        __syncthreads();
        part[t] += add;
        __syncthreads();
    }
    uint64_t acc = t + 1 < kT ? part[t + 1] : 0;  // everything above this segment
    for (int64_t d = hi - 1; d >= lo; --d) {
        if (d <= D) acc += (uint64_t)d * hist[d * k + i];
        TS[d * k + i] = acc;
    }
}

__global__ void k_nw_finalize(NwFinal F)
{
    const uint64_t td = F.tau[1];
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < F.n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = F.sidx[v];
        double s0, s1;
        if (i >= 0) {
            s0 = s1 = (double)F.S[i];
        } else {
            s0 = (double)F.wsum[v] / (double)td;
            s1 = 0.0;
            if (F.hybrid) {
                // first distance beyond the threshold: d a > Delta b
                const uint64_t dmin = (uint64_t)F.delta[v] * F.b / F.a + 1;
                const uint64_t Hs =
                    dmin <= (uint64_t)F.D + 1 ? F.TS[dmin * F.k + F.pivot[v]] : 0;
                const u128 N = (u128)td * (Hs + F.lc[2 * v + 1]) + F.lc[2 * v];
                s1 = u128_to_double(N) / (double)td;
            }
        }
        const double wv = (double)(F.B - F.beta[v]);
        if (F.s_hat[0]) F.s_hat[0][v] = s0;
        if (F.clo[0]) F.clo[0][v] = wv / s0;
        if (F.hybrid) {
            if (F.s_hat[1]) F.s_hat[1][v] = s1;
            if (F.clo[1]) F.clo[1][v] = wv / s1;
        }
    }
}

#define NW_CK(x)                   \
    do {                           \
        if ((x) != cudaSuccess) {  \
            cudaGetLastError();    \
            return CC_ERR_CUDA;    \
        }                          \
    } while (0)
#define NW_RC(x)                     \
    do {                             \
        int r_ = (x);                \
        if (r_ != CC_OK) return r_;  \
    } while (0)

}  // namespace

int nw_total(const uint32_t *beta, int64_t n, uint64_t *dsum, uint64_t *total,
             cudaStream_t st)
{
    NW_CK(cudaMemsetAsync(dsum, 0, 8, st));
    k_total<<<grid_for(n), kT, 0, st>>>(beta, n, reinterpret_cast<unsigned long long *>(dsum));
    NW_CK(cudaGetLastError());
    NW_CK(cudaMemcpyAsync(total, dsum, 8, cudaMemcpyDeviceToHost, st));
    NW_CK(cudaStreamSynchronize(st));
    return CC_OK;
}

int nw_threshold(const uint32_t *beta, int64_t n, int k, uint64_t *keys, uint32_t *vals,
                 uint64_t *tk, uint32_t *tv, uint64_t *pre, uint64_t *tau4, cudaStream_t st)
{
    const int g = grid_for(n);
    k_desc_keys<<<g, kT, 0, st>>>(beta, n, keys, vals);
    bool in_tmp = false;
    NW_RC(device_radix_sort(keys, vals, n, 32, tk, tv, st, &in_tmp));
    uint64_t *sorted = in_tmp ? tk : keys, *b = in_tmp ? keys : tk;
    k_key_to_weight<<<g, kT, 0, st>>>(sorted, n, b);
    uint64_t total = 0;
    NW_RC(device_scan_u64(b, pre, n, &total, st));
    const uint64_t init[4] = {0, 0, 0, (uint64_t)k};
    NW_CK(cudaMemcpyAsync(tau4, init, sizeof(init), cudaMemcpyHostToDevice, st));
    k_tau_test<<<g, kT, 0, st>>>(b, pre, n, k, total,
                                 reinterpret_cast<unsigned long long *>(tau4));
    k_tau_final<<<1, 1, 0, st>>>(b, pre, k, total, tau4);
    NW_CK(cudaGetLastError());
    NW_CK(cudaStreamSynchronize(st));
    return CC_OK;
}

int random_order(int64_t n, uint64_t seed, uint64_t *keys, uint32_t *vals, uint64_t *tk,
                 uint32_t *tv, bool *in_tmp, cudaStream_t st)
{
    k_order_keys<<<grid_for(n), kT, 0, st>>>(n, seed, keys, vals);
    NW_CK(cudaGetLastError());
    return device_radix_sort(keys, vals, n, 64, tk, tv, st, in_tmp);
}

int nw_draw(const uint32_t *beta, int64_t n, int k, uint64_t seed, const uint64_t *tau,
            uint64_t *keys, uint32_t *vals, uint64_t *tk, uint32_t *tv, uint64_t *pre,
            uint64_t *flags, int32_t *out, int64_t *count, cudaStream_t st)
{
    const int g = grid_for(n);
    bool in_tmp = false;
    NW_RC(random_order(n, seed, keys, vals, tk, tv, &in_tmp, st));
    const uint32_t *order = in_tmp ? tv : vals;
    uint64_t *pos = in_tmp ? keys : tk;  // the key buffer not holding the result
    k_lengths<<<g, kT, 0, st>>>(order, beta, tau, n, pre);
    uint64_t line = 0;
    NW_RC(device_scan_u64(pre, pre, n, &line, st));
    k_pick<<<g, kT, 0, st>>>(order, beta, tau, pre, n, seed, flags);
    uint64_t picked = 0;
    NW_RC(device_scan_u64(flags, pos, n, &picked, st));
    k_gather_picked<<<g, kT, 0, st>>>(order, flags, pos, n, k, out);
    NW_CK(cudaGetLastError());
    NW_CK(cudaStreamSynchronize(st));
    *count = (int64_t)picked;
    return CC_OK;
}

void run_nw_mu(int k, const int32_t *sources, const uint32_t *beta, const uint64_t *tau,
               uint32_t *bsrc, uint64_t *mu, unsigned long long *msum, cudaStream_t st)
{
    k_mu<<<(k + kT - 1) / kT, kT, 0, st>>>(k, sources, beta, tau, bsrc, mu, msum);
}

static int grid_tiles(int64_t n)  // a warp per kTile nodes
{
    const int64_t warps = (n + kTile - 1) / kTile;
    return (int)std::min<int64_t>(std::max<int64_t>(1, (warps * 32 + kT - 1) / kT), 152 * 16);
}

void run_nw_reduce1(const NwJob &j, cudaStream_t st)
{
    k_nw_reduce1<<<grid_tiles(j.n), kT, 0, st>>>(j);
}

void run_nw_reduce2(const NwJob &j, int64_t D, cudaStream_t st)
{
    const size_t smem = D < kSmemRows ? (size_t)(D + 1) * 32 * 8 : 0;  // <= 48 KB
    k_nw_reduce2<<<grid_tiles(j.n), kT, smem, st>>>(j, D);
}

void run_nw_tail(const unsigned long long *hist, int64_t D, int k, uint64_t *TS,
                 cudaStream_t st)
{
    k_nw_tail<<<k, kT, 0, st>>>(hist, D, k, TS);
}

void run_nw_finalize(const NwFinal &f, cudaStream_t st)
{
    k_nw_finalize<<<grid_for(f.n), kT, 0, st>>>(f);
}

}  // namespace ccg
