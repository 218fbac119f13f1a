// Outbound / inbound estimates of general directed graphs (section 6.2,
// Algorithm 4): for every node v, the k nodes of smallest rank (a seeded
// random order) among those v reaches (outbound) or that reach v (inbound),
// their distances, and the rank position of the k-th.
//
// One persistent cooperative launch walks the order in groups of 64 W
// sources.  Each group is a bit-packed multi-source BFS on the search graph
// (G^T for outbound, G for inbound: bit i leaves the group's i-th source),
// recording the level at which each bit first reaches each node; then every
// node it touched accepts its lowest-rank bits (its own excluded) until it
// holds k samples.  Bits are ranks, so the accepted ones are exactly the
// next samples in rank order.
//
// Pruning: a node x saturated at the start of a group -- k + 1 sources
// other than x have reached it, or k have and x's own search has run --
// holds k + 1 nodes of smaller rank than every source still to come among
// x and its reachability set; every node that reaches x through x holds k
// of them other than itself, so x is neither entered nor expanded.  Nodes
// that saturate during a group still propagate that group's bits: extra
// bits only reach nodes that really reach the source, and each node keeps
// its lowest ranks, so the samples equal those of the sequential procedure
// with this pruning, and the first-arrival levels are exact distances
// (every node on a shortest path from v to an accepted source is
// unsaturated).  Algorithm 4 prunes at k nodes other than x, which can stop
// a search at a node whose k samples include v and leave v a sample short;
// the rule above keeps the stated aim, a uniform sample of size k of every
// reachability set.
//
// With arc lengths (section 6.2 runs Dijkstra) each (node, source) slot
// holds a tentative distance instead of a level: a round relaxes every
// source whose distance at a frontier node dropped into its neighbours
// (atomicMin), the nodes that improved form the next frontier, and the
// rounds end when nothing improves -- label-correcting search, exact on the
// unsaturated nodes by the same argument.  The slots of a node return to
// infinity when it takes its samples.
//
// Every wait is the bounded grid barrier (CC_ERR_TIMEOUT on expiry).
#include <algorithm>
#include <cstdint>
#include <cstring>

#include "barrier.cuh"
#include "nodew.h"
#include "reach.h"

namespace ccg {

namespace {

constexpr int kRT = 256;

struct RState {
    unsigned qlen[2];
    unsigned tlen[2];
    unsigned long long levels, groups, pushes;
};

__device__ __forceinline__ bool saturated(const ReachJob &J, int32_t x, int64_t base)
{
    const int c = J.cnt[x];
    return c >= J.k && (J.extra[x] || (int64_t)J.rank[x] < base);
}

__global__ void __launch_bounds__(kRT, 4) k_reach(ReachJob J, RState *rs)
{
    const unsigned nb = gridDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int64_t gw = tid >> 5, nwarps = nthr >> 5;
    const int W = J.W, G = 64 * W;
    volatile unsigned *qlen = rs->qlen, *tlen = rs->tlen;
    unsigned epoch = 0;
    int par = 0;
    for (int64_t base = 0; base < J.n; base += G, par ^= 1) {
        const int gs = (int)(J.n - base < G ? J.n - base : G);
        int cur = 0;
        // sources of the group (distinct nodes: one thread each)
        for (int64_t i = tid; i < gs; i += nthr) {
            const int32_t s = J.order[base + i];
            if (saturated(J, s, base)) continue;
            const uint64_t bit = 1ull << (i & 63);
            J.vis[(int64_t)s * W + (i >> 6)] = bit;
            J.F[(int64_t)s * W + (i >> 6)] = bit;
            J.lev[(int64_t)s * G + i] = 0;
            J.Q[0][atomicAdd((unsigned *)&qlen[0], 1u)] = s;
            J.TL[atomicAdd((unsigned *)&tlen[par], 1u)] = s;
        }
        if (!grid_sync(J.ctl, blockIdx.x, nb, J.timeout_ns)) return;
        uint32_t level = 0;
        for (;;) {
            const unsigned qn = qlen[cur];
            if (qn == 0) break;
            ++level;
            ++epoch;
            const int nxq = cur ^ 1;
            // expand: a warp per frontier node, a lane per arc
            for (int64_t idx = gw; idx < qn; idx += nwarps) {
                const int32_t u = J.Q[cur][idx];
                uint64_t Fu[kReachMaxW];
#pragma unroll
                for (int q = 0; q < kReachMaxW; ++q)
                    Fu[q] = q < W ? J.F[(int64_t)u * W + q] : 0;
                for (int64_t e = J.rp[u] + lane; e < J.rp[u + 1]; e += 32) {
                    const int32_t w = J.col[e];
                    if (saturated(J, w, base)) continue;
                    bool any = false;
                    if (J.w) {
                        // arc lengths: relax every changed source of u into w
                        const uint64_t len = J.w[e];
#pragma unroll
                        for (int q = 0; q < kReachMaxW; ++q) {
                            if (q >= W) break;
                            uint64_t imp = 0;
                            for (uint64_t x = Fu[q]; x; x &= x - 1) {
                                const int i = q * 64 + (__ffsll((long long)x) - 1);
                                const uint64_t cand =
                                    (uint64_t)__ldcg(&J.lev[(int64_t)u * G + i]) + len;
                                if (cand >= (uint64_t)kInf) continue;
                                const uint32_t old =
                                    atomicMin(&J.lev[(int64_t)w * G + i], (uint32_t)cand);
                                if (cand < old) imp |= 1ull << (i & 63);
                            }
                            if (imp) {
                                atomicOr((unsigned long long *)&J.nxt[(int64_t)w * W + q],
                                         (unsigned long long)imp);
                                any = true;
                            }
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < kReachMaxW; ++q) {
                            if (q >= W) break;
                            const uint64_t nbits = Fu[q] & ~J.vis[(int64_t)w * W + q];
                            if (nbits) {
                                atomicOr((unsigned long long *)&J.nxt[(int64_t)w * W + q],
                                         (unsigned long long)nbits);
                                any = true;
                            }
                        }
                    }
                    if (any && atomicExch(&J.qstamp[w], epoch) != epoch)
                        J.Q[nxq][atomicAdd((unsigned *)&qlen[nxq], 1u)] = w;
                }
            }
            if (!grid_sync(J.ctl, blockIdx.x, nb, J.timeout_ns)) return;
            // the next frontier: new bits (with arc lengths: the sources whose
            // distance dropped), their levels, first touches
            const unsigned qn2 = qlen[nxq];
            for (int64_t idx = tid; idx < qn2; idx += nthr) {
                const int32_t w = J.Q[nxq][idx];
                bool fresh = true;
                for (int q = 0; q < W; ++q) {
                    const int64_t at = (int64_t)w * W + q;
                    const uint64_t old = J.vis[at];
                    const uint64_t nbits = J.w ? J.nxt[at] : J.nxt[at] & ~old;
                    if (old) fresh = false;
                    J.nxt[at] = 0;
                    J.vis[at] = old | nbits;
                    J.F[at] = nbits;
                    if (!J.w)
                        for (uint64_t x = nbits; x; x &= x - 1)
                            J.lev[(int64_t)w * G + q * 64 + (__ffsll((long long)x) - 1)] = level;
                }
                if (fresh) J.TL[atomicAdd((unsigned *)&tlen[par], 1u)] = w;
            }
            if (tid == 0) {
                qlen[cur] = 0;
                atomicAdd(&rs->levels, 1ull);
            }
            cur = nxq;
            if (!grid_sync(J.ctl, blockIdx.x, nb, J.timeout_ns)) return;
        }
        // acceptance: each touched node takes its lowest-rank bits
        const unsigned tn = tlen[par];
        for (int64_t idx = tid; idx < tn; idx += nthr) {
            const int32_t v = J.TL[idx];
            const int64_t rv = J.rank[v];
            int c = J.cnt[v];
            uint64_t ds = J.dsum[v];
            bool done = false;
            for (int q = 0; q < W; ++q) {
                const int64_t at = (int64_t)v * W + q;
                const uint64_t reached = J.vis[at];
                uint64_t bits = reached;
                J.vis[at] = 0;
                J.F[at] = 0;
                if (rv >= base && rv < base + gs && (rv - base) >> 6 == q)
                    bits &= ~(1ull << ((rv - base) & 63));  // its own search
                for (; bits && !done; bits &= bits - 1) {
                    const int i = q * 64 + (__ffsll((long long)bits) - 1);
                    if (c < J.k) {
                        ds += J.lev[(int64_t)v * G + i];
                        if (++c == J.k) {
                            const int64_t t = base + i + 1;  // 1-based rank position
                            J.T[v] = rv < base + i ? t - 1 : t;
                        }
                    } else {
                        J.extra[v] = 1;  // a (k+1)-th source reached v
                        done = true;
                    }
                }
                if (J.w)  // tentative distances start at infinity in every group
                    for (uint64_t x = reached; x; x &= x - 1)
                        J.lev[(int64_t)v * G + q * 64 + (__ffsll((long long)x) - 1)] = kInf;
            }
            J.cnt[v] = c;
            J.dsum[v] = ds;
        }
        if (tid == 0) {
            tlen[par ^ 1] = 0;  // the next group's touched list
            rs->groups += 1;
        }
        if (!grid_sync(J.ctl, blockIdx.x, nb, J.timeout_ns)) return;
        if (tid == 0) tlen[par] = 0;  // read by every CTA before the barrier
    }
}

__global__ void k_rank_of(const uint32_t *order, int64_t n, int32_t *order32, int32_t *rank)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = order[p];
        order32[p] = (int32_t)v;
        rank[v] = (int32_t)p;
    }
}

__global__ void k_reach_final(int64_t n, int k, const int32_t *cnt, const uint64_t *dsum,
                              const int64_t *T, double *avg, double *rhat)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int c = cnt[v];
        if (avg) avg[v] = c ? (double)dsum[v] / (double)c : 0.0;
        if (rhat) {
            double r = (double)c;
            if (c >= k)
                r = k == 1 ? 1.0
                           : 1.0 + (double)((uint64_t)(k - 1) * (uint64_t)(n - 2)) /
                                       (double)(T[v] - 1);
            rhat[v] = r;
        }
    }
}

int grid_of(int64_t n)
{
    return (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 152 * 16);
}

#define R_CK(x)                                  \
    do {                                         \
        const cudaError_t e_ = (x);              \
        if (e_ != cudaSuccess) {                 \
            note_cuda_error(e_, __FILE__, __LINE__); \
            cudaGetLastError();                  \
            return CC_ERR_CUDA;                  \
        }                                        \
    } while (0)
#define R_RC(x)                      \
    do {                             \
        int r_ = (x);                \
        if (r_ != CC_OK) return r_;  \
    } while (0)

}  // namespace

int reach_order(int64_t n, uint64_t seed, uint64_t *keys, uint32_t *vals, uint64_t *tk,
                uint32_t *tv, int32_t *order, int32_t *rank, cudaStream_t st)
{
    bool in_tmp = false;
    R_RC(random_order(n, seed, keys, vals, tk, tv, &in_tmp, st));
    k_rank_of<<<grid_of(n), 256, 0, st>>>(in_tmp ? tv : vals, n, order, rank);
    R_CK(cudaGetLastError());
    return CC_OK;
}

int reach_run(const ReachJob &job, cudaStream_t st, ReachStats *stats)
{
    int dev = 0, sms = 0, per = 0;
    R_CK(cudaGetDevice(&dev));
    R_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    R_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_reach, kRT, 0));
    if (per < 1) return CC_ERR_CUDA;
    int grid = sms * std::min(per, 4);
    RState *rs = nullptr;
    R_CK(cudaMallocAsync((void **)&rs, sizeof(RState), st));
    int rc = CC_OK;
    if (cudaMemsetAsync(rs, 0, sizeof(RState), st) != cudaSuccess ||
        cudaMemsetAsync(job.ctl, 0, sizeof(Ctl), st) != cudaSuccess) {
        rc = CC_ERR_CUDA;
    } else {
        ReachJob j = job;
        void *args[] = {(void *)&j, (void *)&rs};
        if (cudaLaunchCooperativeKernel((const void *)k_reach, grid, kRT, args, 0, st) !=
            cudaSuccess)
            rc = CC_ERR_CUDA;
    }
    RState h{};
    Ctl c{};
    if (rc == CC_OK && (cudaMemcpyAsync(&h, rs, sizeof(h), cudaMemcpyDeviceToHost, st) !=
                            cudaSuccess ||
                        cudaMemcpyAsync(&c, job.ctl, sizeof(c), cudaMemcpyDeviceToHost, st) !=
                            cudaSuccess ||
                        cudaStreamSynchronize(st) != cudaSuccess))
        rc = CC_ERR_CUDA;
    cudaFreeAsync(rs, st);
    if (rc != CC_OK) {
        cudaGetLastError();
        return rc;
    }
    if (stats) {
        stats->levels = (int64_t)h.levels;
        stats->groups = (int64_t)h.groups;
        stats->grid = grid;
    }
    return c.err < 0 ? c.err : CC_OK;
}

void reach_finalize(int64_t n, int k, const int32_t *cnt, const uint64_t *dsum,
                    const int64_t *T, double *avg, double *rhat, cudaStream_t st)
{
    k_reach_final<<<grid_of(n), 256, 0, st>>>(n, k, cnt, dsum, T, avg, rhat);
}

}  // namespace ccg
