// Multi-source shortest paths with uint32 arc lengths, 32 sources at a time
// (sections 3 and 7: one Dijkstra per sampled node, 32-bit integer arc
// lengths), and the per-chunk reductions that feed the same estimators as the
// breadth-first path.  The rounds relax by buckets of distance (delta-
// stepping): see mssp_kernel.
//
// A chunk holds the tentative distances of up to 32 sources as one 128-byte
// row per node (dist[v][lane], lane = source within the chunk), so a warp
// owns a node and each lane one source: every row read or atomicMin is one
// coalesced line.  The chunk is solved by label-correcting relaxation in
// rounds (Bellman-Ford over an active-node queue): a node is queued when
// some source's distance to it drops, with a per-node bit mask of the
// sources whose distance dropped; a round relaxes the out-arcs of every
// queued node for exactly those sources.  Rounds run inside one persistent
// cooperative kernel separated by a bounded grid barrier.
//
// Directed round-trip distances (section 6.1) are the sum of a chunk solved
// on G and the same chunk solved on the reversed graph; the reductions take
// either one distance matrix or the pair.
#include <cstdint>

#include "barrier.cuh"
#include "cc_internal.h"
#include "sssp.h"

namespace ccg {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
// Arcs of a queued node relaxed together: their column indices, lengths,
// neighbour labels and atomicMins are each in flight at once, so a node
// of a few arcs costs one chain of dependent accesses, not one per arc.
#ifndef CC_MSSP_ARCS
#define CC_MSSP_ARCS 3
#endif
#ifndef CC_MSSP_MIN_CTAS
#define CC_MSSP_MIN_CTAS 4
#endif
constexpr int kArcs = CC_MSSP_ARCS;

// Sources per row: 32 * SPL (SPL = 1 or 2), lane l holding sources l and
// l + 32 of the chunk; masks are 64-bit either way.
template <int SPL>
__global__ void __launch_bounds__(kBlock, CC_MSSP_MIN_CTAS) mssp_kernel(SsspJob J)
{
    constexpr int LD = 32 * SPL;  // row stride
    const int lane = threadIdx.x & 31;
    const int64_t gthreads = (int64_t)gridDim.x * kBlock;
    const int64_t gtid = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    const int64_t gwarp = gtid >> 5, nwarps = gthreads >> 5;
    const int64_t n = J.n;
    Ctl *ctl = J.ctl;
    const unsigned nb = gridDim.x;
    unsigned long long relax = 0;
    __shared__ int32_t s_buf[kStage], s_fbuf[kStage];
    __shared__ unsigned s_cnt, s_base, s_fcnt, s_fbase;
    const Stage stage{s_buf, &s_cnt, &s_base};
    const Stage fstage{s_fbuf, &s_fcnt, &s_fbase};
    if (threadIdx.x == 0) {
        s_cnt = 0;
        s_fcnt = 0;
    }

    if (gtid < 3) ctl->far_min[gtid] = ~0ull;
    for (int64_t i = gtid; i < n * LD; i += gthreads) J.dist[i] = kInf;
    for (int64_t v = gtid; v < n; v += gthreads) {
        J.mask[v] = 0ull;
        if (J.delta) {
            J.nstamp[v] = 0u;
            J.fstamp[v] = 0u;
        }
    }
    if (!grid_sync(ctl, blockIdx.x, nb, J.timeout_ns)) return;
    if (gtid < J.kc) {
        const int v = J.sources[gtid];
        J.dist[(int64_t)v * LD + gtid] = 0u;
        if (atomicOr(&J.mask[v], 1ull << gtid) == 0ull) {
            const unsigned p = atomicAdd(&ctl->lev[0].qlen, 1u);
            J.Q0[p] = v;
            if (J.delta) J.nstamp[v] = 1u;  // queued for round 0
        }
    }
    if (!grid_sync(ctl, blockIdx.x, nb, J.timeout_ns)) return;

    // Epoch e fills far queue e % 3; at the advance to e + 1 that queue is
    // processed as the round's queue and queue (e + 2) % 3, consumed two
    // advances ago, gets its length cleared for epoch e + 2.
    const uint64_t delta = J.delta;
    uint64_t T = delta ? delta : ~0ull;
    unsigned epoch = 0;
    int r = 0;
    for (;; ++r) {
        unsigned qn = ((volatile LevelCtl *)&ctl->lev[r & 3])->qlen;
        const int32_t *Qin = (r & 1) ? J.Q1 : J.Q0;
        if (qn == 0) {
            if (!delta) break;
            const unsigned fn = ((volatile Ctl *)ctl)->far_len[epoch % 3];
            if (fn == 0) break;
            Qin = J.far[epoch % 3];
            qn = fn;
            // next bucket: at least one step, and on to the one holding the
            // smallest waiting label (empty buckets are skipped)
            const unsigned long long fmin = ((volatile Ctl *)ctl)->far_min[epoch % 3];
            T += delta;
            if (fmin != ~0ull && fmin >= T) T = (fmin / delta + 1) * delta;
            epoch += 1;
            if (gtid == 0) {
                ctl->far_len[(epoch + 1) % 3] = 0;
                ctl->far_min[(epoch + 1) % 3] = ~0ull;
                ctl->td_levels += 1;
            }
        }
        if (gtid == 0) ((LevelCtl *)&ctl->lev[(r + 2) & 3])->qlen = 0;
        int32_t *Qout = (r & 1) ? J.Q0 : J.Q1;
        unsigned *qout_len = &ctl->lev[(r + 1) & 3].qlen;
        int32_t *Fout = delta ? J.far[epoch % 3] : nullptr;
        unsigned *fout_len = &ctl->far_len[epoch % 3];
        const unsigned nst = (unsigned)r + 2u;  // stamp: queued for round r + 1
        const unsigned fst = epoch + 1u;        // stamp: in this epoch's far queue
        for (int64_t t = gwarp; t < (int64_t)qn; t += nwarps) {
            const int u = Qin[t];
            // the row offsets do not depend on the mask: in flight with it
            const int64_t b = J.rp[u], e = J.rp[u + 1];
            unsigned long long m = 0;
            if (lane == 0) m = atomicExch(&J.mask[u], 0ull);
            m = __shfl_sync(FULL, m, 0);
            // The row may have been lowered by an atomicMin of another SM in
            // this round (that is what set the mask bit): read it from L2,
            // the point where those atomics are performed, not from a
            // possibly stale L1 line.  Labels at or beyond the threshold
            // wait in the far queue.
            uint64_t du[SPL];
            bool active[SPL];
            unsigned long long later = 0, lo = ~0ull;
#pragma unroll
            for (int q = 0; q < SPL; ++q) {
                const int i = lane + 32 * q;
                const bool pending = (m >> i) & 1ull;
                du[q] = pending ? __ldcg(J.dist + (int64_t)u * LD + i) : 0ull;
                active[q] = pending && du[q] < T;
                const unsigned bl = __ballot_sync(FULL, pending && !active[q]);
                later |= (unsigned long long)bl << (32 * q);
                if (pending && !active[q]) lo = du[q] < lo ? du[q] : lo;
            }
            if (later) {
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) {
                    const unsigned long long y = __shfl_xor_sync(FULL, lo, o);
                    lo = y < lo ? y : lo;
                }
                if (lane == 0) {
                    atomicOr(&J.mask[u], later);
                    atomicMin(&ctl->far_min[epoch % 3], lo);
                    if (atomicExch(&J.fstamp[u], fst) != fst)
                        stage_push(fstage, u, Fout, fout_len);
                }
            }
            bool any = false;
#pragma unroll
            for (int q = 0; q < SPL; ++q) any |= active[q];
            if (!__any_sync(FULL, any)) continue;
            for (int64_t x0 = b; x0 < e; x0 += kArcs) {
                int vv[kArcs];
                uint32_t wt[kArcs];
#pragma unroll
                for (int j = 0; j < kArcs; ++j) {
                    const int64_t x = x0 + j;
                    vv[j] = x < e ? __ldg(J.col + x) : -1;
                    wt[j] = x < e && J.w ? __ldg(J.w + x) : 1u;
                }
                // Neighbour labels (a possibly stale L1 copy only lets more
                // candidates through: labels only fall), then the atomicMins
                // of every candidate: imp bit j * SPL + q = label improved.
                unsigned cur[kArcs][SPL];
#pragma unroll
                for (int j = 0; j < kArcs; ++j)
#pragma unroll
                    for (int q = 0; q < SPL; ++q)
                        cur[j][q] = vv[j] >= 0 && active[q]
                                        ? J.dist[(int64_t)vv[j] * LD + lane + 32 * q]
                                        : 0u;
                unsigned imp = 0;
#pragma unroll
                for (int j = 0; j < kArcs; ++j)
#pragma unroll
                    for (int q = 0; q < SPL; ++q) {
                        if (vv[j] < 0 || !active[q]) continue;
                        const uint64_t nd = du[q] + wt[j];
                        relax += 1;
                        if (nd >= (uint64_t)kInf) {
                            atomicCAS(&ctl->err, 0, CC_ERR_TOO_LARGE);
                        } else if ((unsigned)nd < cur[j][q]) {
                            unsigned *slot = &J.dist[(int64_t)vv[j] * LD + lane + 32 * q];
                            if ((unsigned)nd < atomicMin(slot, (unsigned)nd))
                                imp |= 1u << (j * SPL + q);
                        }
                    }
#pragma unroll
                for (int j = 0; j < kArcs; ++j) {
                    if (vv[j] < 0) break;  // uniform over the warp
                    const int v = vv[j];
                    unsigned long long nbits = 0, fbits = 0, flo = ~0ull;
#pragma unroll
                    for (int q = 0; q < SPL; ++q) {
                        const bool im = (imp >> (j * SPL + q)) & 1u;
                        const uint64_t nd = du[q] + wt[j];
                        nbits |= (unsigned long long)__ballot_sync(FULL, im && nd < T) << (32 * q);
                        fbits |= (unsigned long long)__ballot_sync(FULL, im && nd >= T) << (32 * q);
                        if (im && nd >= T) flo = nd < flo ? nd : flo;
                    }
                    if (!(nbits | fbits)) continue;
                    if (!delta) {  // no buckets: one queue
                        if (lane == 0 && atomicOr(&J.mask[v], nbits | fbits) == 0ull)
                            stage_push(stage, v, Qout, qout_len);
                        continue;
                    }
                    if (fbits) {
#pragma unroll
                        for (int o = 16; o >= 1; o >>= 1) {
                            const unsigned long long y = __shfl_xor_sync(FULL, flo, o);
                            flo = y < flo ? y : flo;
                        }
                    }
                    if (lane == 0) {
                        atomicOr(&J.mask[v], nbits | fbits);
                        if (nbits && atomicExch(&J.nstamp[v], nst) != nst)
                            stage_push(stage, v, Qout, qout_len);
                        if (fbits) {
                            atomicMin(&ctl->far_min[epoch % 3], flo);
                            if (atomicExch(&J.fstamp[v], fst) != fst)
                                stage_push(fstage, v, Fout, fout_len);
                        }
                    }
                }
            }
        }
        stage_flush(stage, Qout, qout_len);
        if (delta) stage_flush(fstage, Fout, fout_len);
        if (!grid_sync(ctl, blockIdx.x, nb, J.timeout_ns)) return;
    }
    __shared__ unsigned long long s_rel[kBlock / 32];
    for (int o = 16; o >= 1; o >>= 1) relax += __shfl_xor_sync(FULL, relax, o);
    if (lane == 0) s_rel[threadIdx.x >> 5] = relax;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < kBlock / 32; ++i) t += s_rel[i];
        atomicAdd(&ctl->words, t);
    }
    if (gtid == 0) ctl->levels = r;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

// Distance of the lane's source to v in this chunk (round trip when a
// reverse matrix is given); kInf when unreachable or not a source lane.
__device__ __forceinline__ uint64_t chunk_dist(const ReduceJob &R, int64_t v, int lane)
{
    if (lane >= R.kc) return (uint64_t)kInf;
    const int64_t r = R.row_of ? (int64_t)R.row_of[v] : v;
    const uint64_t a = R.distF[r * R.ld + R.sub + lane];
    if (!R.distR) return a;
    const uint64_t b = R.distR[r * R.ld + R.sub + lane];
    if (a == kInf || b == kInf) return (uint64_t)kInf;
    return a + b;
}

// Pass-1 reduction of one chunk: sums, running (distance, index) minimum
// for the pivot, distances between sampled nodes, exact S of the chunk's
// sources and the largest distance.  A warp takes kTile nodes at a time,
// lane = source: the rows of all kTile nodes are loaded before any is
// reduced (one memory round trip per tile, not per node), and lane u then
// holds node u's sums and key for the read-modify-writes, which the first
// kTile lanes issue together.
constexpr int kTile = 8;

__global__ void k_reduce1(ReduceJob R)
{
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int gi = R.base + lane;
    const bool valid = lane < R.kc;
    unsigned long long Sl = 0, dmax = 0;
    int bad = 0;
    for (int64_t v0 = gwarp * kTile; v0 < R.n; v0 += nwarps * kTile) {
        uint64_t d[kTile];
#pragma unroll
        for (int u = 0; u < kTile; ++u)
            d[u] = v0 + u < R.n ? chunk_dist(R, v0 + u, lane) : (uint64_t)kInf;
        const int32_t sx =
            !R.sum_only && lane < kTile && v0 + lane < R.n ? R.sidx[v0 + lane] : -1;
        unsigned long long my_s = 0, my_s2 = 0, my_key = ~0ull;
#pragma unroll
        for (int u = 0; u < kTile; ++u) {
            if (v0 + u >= R.n) break;  // warp-uniform
            const uint64_t du = d[u];
            if (valid && du >= (uint64_t)kInf) bad = 1;
            const uint64_t dd = valid && du < kInf ? du : 0;
            Sl += dd;
            dmax = dd > dmax ? dd : dmax;
            const unsigned long long s = warp_sum(dd), s2 = warp_sum(dd * dd);
            unsigned long long key = valid ? ((du << 32) | (uint64_t)gi) : ~0ull;
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(FULL, key, o);
                key = y < key ? y : key;
            }
            if (lane == u) {
                my_s = s;
                my_s2 = s2;
                my_key = key;
            }
            const int j = __shfl_sync(FULL, sx, u);
            if (j >= 0 && valid) R.dcc[(int64_t)gi * R.k + j] = (uint32_t)dd;
        }
        if (lane < kTile && v0 + lane < R.n) {
            const int64_t v = v0 + lane;
            R.sum2[2 * v] += my_s;
            R.sum2[2 * v + 1] += my_s2;
            if (!R.sum_only && my_key < R.best[v]) R.best[v] = my_key;
        }
    }
    // Per-source sums and the largest distance are combined over the CTA in
    // shared memory first: one global atomic per (CTA, source), not per
    // (warp, source), and one atomicMax per CTA (same-address atomics from
    // every lane serialise in L2).
    __shared__ unsigned long long s_S[kBlock / 32][32], s_max[kBlock / 32];
    const int wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(FULL, dmax, o);
        dmax = y > dmax ? y : dmax;
    }
    s_S[wid][lane] = Sl;
    if (lane == 0) s_max[wid] = dmax;
    __syncthreads();
    if (threadIdx.x < 32 && !R.sum_only) {
        unsigned long long t = 0, m = 0;
        for (int w = 0; w < kBlock / 32; ++w) {
            t += s_S[w][threadIdx.x];
            m = s_max[w] > m ? s_max[w] : m;
        }
        if (threadIdx.x < R.kc && t) atomicAdd(&R.S_samp[R.base + threadIdx.x], t);
        if (threadIdx.x == 0 && m) atomicMax(R.dmax, m);
    }
    if (bad) atomicExch(R.err, CC_ERR_DISCONNECTED);
}

// Pass-2 reduction of one chunk for the hybrid estimator: per-source
// distance histogram over V \ C and the sums over the sources in L(v).
// The histogram of this chunk's columns is accumulated per CTA in shared
// memory when the distances are small (D < kSmemHistRows), then added to the
// global one: many nodes share a (distance, source) cell.
constexpr int kSmemHistRows = 256;

__global__ void k_reduce2(ReduceJob R)
{
    extern __shared__ unsigned sh[];  // (D+1) x 32 when D < kSmemHistRows
    const bool local = R.D < kSmemHistRows;
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int gi = R.base + lane;
    if (local) {
        for (int i = threadIdx.x; i < (R.D + 1) * 32; i += blockDim.x) sh[i] = 0u;
        __syncthreads();
    }
    for (int64_t v = gwarp; v < R.n; v += nwarps) {
        if (R.sidx[v] >= 0) continue;
        const bool valid = lane < R.kc;
        const uint64_t d = valid ? chunk_dist(R, v, lane) : 0;
        if (valid) {
            if (local) atomicAdd(&sh[d * 32 + lane], 1u);
            else atomicAdd(&R.hist[(int64_t)d * R.k + gi], 1u);
        }
        bool inL = false;
        if (valid) {
            const uint64_t m = R.Lmask[v * R.W + (gi >> 6)];
            inL = (m >> (gi & 63)) & 1ull;
        }
        const unsigned long long s = warp_sum(inL ? d : 0), s2 = warp_sum(inL ? d * d : 0);
        if (lane == 0 && s) {
            R.lc2[2 * v] += s;
            R.lc2[2 * v + 1] += s2;
        }
        const uint8_t f = R.sqflag ? R.sqflag[v] : 0;
        if (f) {
            const int p = R.pivot[v];
            if (f & 1) {
                // 128-bit warp sum of the squared errors of this chunk's
                // sources beyond the threshold.
                uint64_t lo = 0, hi = 0;
                if (valid && !inL) {
                    const int64_t e = (int64_t)d - (int64_t)R.dcc[(int64_t)p * R.k + gi];
                    const uint64_t ae = (uint64_t)(e < 0 ? -e : e);
                    lo = ae * ae;
                }
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) {
                    const uint64_t olo = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
                    const uint64_t ohi = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
                    const uint64_t nlo = lo + olo;
                    hi += ohi + (nlo < lo ? 1u : 0u);
                    lo = nlo;
                }
                if (lane == 0 && (lo | hi)) {
                    const uint64_t nlo = R.hcse[2 * v] + lo;
                    R.hcse[2 * v + 1] += hi + (nlo < lo ? 1u : 0u);
                    R.hcse[2 * v] = nlo;
                }
            }
            if ((f & 2) && valid && gi == R.istar[p]) R.fdist[v] = (uint32_t)d;
        }
    }
    if (local) {
        __syncthreads();
        for (int i = threadIdx.x; i < (R.D + 1) * 32; i += blockDim.x) {
            const int l = i >> 5, c = i & 31;
            if (c < R.kc && sh[i]) atomicAdd(&R.hist[(int64_t)l * R.k + R.base + c], sh[i]);
        }
    }
}

// best[v] = (Delta << 32 | pivot index)  ->  pivot[v], delta[v]
__global__ void k_unpack_pivot(int64_t n, const unsigned long long *best, int32_t *pivot,
                               uint32_t *delta)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        pivot[v] = (int32_t)(best[v] & 0xFFFFFFFFull);
        delta[v] = (uint32_t)(best[v] >> 32);
    }
}

int grid_of(int64_t n)
{
    int64_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

int launch_mssp(const SsspJob &job, cudaStream_t st)
{
    static int blocks_per_sm[2] = {-1, -1}, sms = 0;
    const int q = job.spl == 2 ? 1 : 0;
    const void *fn = q ? (const void *)mssp_kernel<2> : (const void *)mssp_kernel<1>;
    if (blocks_per_sm[q] < 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return CC_ERR_CUDA;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return CC_ERR_CUDA;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm[q], fn, kBlock, 0) !=
                cudaSuccess ||
            blocks_per_sm[q] < 1)
            return CC_ERR_CUDA;
    }
    SsspJob j = job;
    void *args[] = {&j};
    int grid = blocks_per_sm[q] * sms;
    if (job.max_ctas > 0 && job.max_ctas < grid) grid = job.max_ctas;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlock), args, 0, st) == cudaSuccess
               ? CC_OK
               : CC_ERR_CUDA;
}

// One carveout for every persistent kernel of a server (see msbfs.cu).
void mssp_set_carveout(int percent)
{
    for (const void *f : {(const void *)mssp_kernel<1>, (const void *)mssp_kernel<2>})
        cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, percent);
    cudaGetLastError();
}

// Smallest residency over both variants.
int mssp_blocks_per_sm()
{
    int m = 1 << 30;
    for (const void *f : {(const void *)mssp_kernel<1>, (const void *)mssp_kernel<2>}) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, kBlock, 0) != cudaSuccess) {
            cudaGetLastError();
            return 1;
        }
        m = b < m ? b : m;
    }
    return m < 1 ? 1 : m;
}

void run_reduce1(const ReduceJob &r, cudaStream_t st)
{
    k_reduce1<<<grid_of(r.n * 32), kBlock, 0, st>>>(r);
}

void run_reduce2(const ReduceJob &r, cudaStream_t st)
{
    const size_t smem = r.D < kSmemHistRows ? (size_t)(r.D + 1) * 32 * 4 : 0;
    k_reduce2<<<grid_of(r.n * 32), 256, smem, st>>>(r);
}

void run_unpack_pivot(int64_t n, const unsigned long long *best, int32_t *pivot,
                      uint32_t *delta, cudaStream_t st)
{
    k_unpack_pivot<<<grid_of(n), 256, 0, st>>>(n, best, pivot, delta);
}

}  // namespace ccg
