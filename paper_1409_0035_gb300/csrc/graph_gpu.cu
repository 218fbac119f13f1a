// Graph to CSR on the device (undirected graphs): the preprocessing step
// that section 7 counts in its times.
//
//   1. arcs: each edge u-v gives the keys (u << 32 | v) and (v << 32 | u)
//      with its length; self-loops dropped (stream compaction);
//   2. stable LSD radix sort of the 64-bit keys (8-bit digits, only the
//      2 * ceil(log2 n) significant bits), lengths carried along;
//   3. parallel arcs merged keeping the smallest length (segmented minimum
//      over equal keys), then compacted;
//   4. row offsets from the sorted tails;
//   5. connected components by lock-free union-find (roots hooked under the
//      smaller root with atomicCAS, path halving), so a component's label
//      is its smallest node id; the largest component wins, ties to the
//      smallest label;
//   6. kept nodes renumbered in increasing original id (exclusive scan) and
//      the rows rewritten (monotone renumbering keeps them sorted).
#include <algorithm>
#include <cstdint>
#include <vector>

#include "cc_internal.h"
#include "graph_gpu.h"

namespace ccg {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;                 // keys per thread per sort tile
constexpr int kTile = kThreads * kItems;   // 4096 keys per tile
constexpr int kRadix = 256;

// ---------------------------------------------------------------- scan

// Exclusive scan of uint64 values in tiles of kThreads*4: per-tile sums,
// scan of the sums (recursively), then the in-tile scan plus offset.
__global__ void k_tile_sums(const uint64_t *in, int64_t n, uint64_t *sums)
{
    __shared__ uint64_t s[kThreads];
    const int64_t base = (int64_t)blockIdx.x * kThreads * 4;
    uint64_t t = 0;
    for (int j = 0; j < 4; ++j) {
        const int64_t i = base + (int64_t)j * kThreads + threadIdx.x;
        if (i < n) t += in[i];
    }
    s[threadIdx.x] = t;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = s[0];
}

__global__ void k_tile_scan(const uint64_t *in, int64_t n, const uint64_t *offs,
                            uint64_t *out)
{
    __shared__ uint64_t s[kThreads * 4];
    const int64_t base = (int64_t)blockIdx.x * kThreads * 4;
    for (int j = 0; j < 4; ++j) {
        const int64_t i = base + (int64_t)j * kThreads + threadIdx.x;
        s[j * kThreads + threadIdx.x] = i < n ? in[i] : 0;
    }
    __syncthreads();
    // each thread scans 4 consecutive values, then a Hillis-Steele scan of
    // the thread totals
    uint64_t v[4], tot = 0;
    for (int j = 0; j < 4; ++j) {
        v[j] = s[threadIdx.x * 4 + j];
        tot += v[j];
    }
    __shared__ uint64_t t[kThreads];
    t[threadIdx.x] = tot;
    __syncthreads();
    for (int o = 1; o < kThreads; o <<= 1) {
        const uint64_t a = threadIdx.x >= o ? t[threadIdx.x - o] : 0;
        __syncthreads();
        t[threadIdx.x] += a;
        __syncthreads();
    }
    uint64_t run = t[threadIdx.x] - tot + offs[blockIdx.x];
    __syncthreads();
    for (int j = 0; j < 4; ++j) {
        s[threadIdx.x * 4 + j] = run;
        run += v[j];
    }
    __syncthreads();
    for (int j = 0; j < 4; ++j) {
        const int64_t i = base + (int64_t)j * kThreads + threadIdx.x;
        if (i < n) out[i] = s[j * kThreads + threadIdx.x];
    }
}

// ---------------------------------------------------------------- sort

__global__ void k_digit_hist(const uint64_t *keys, int64_t n, int shift, int nbits,
                             uint32_t *counts, int ntiles)
{
    __shared__ uint32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    const uint64_t mask = (1ull << nbits) - 1;
    for (int j = 0; j < kItems; ++j) {
        const int64_t i = base + (int64_t)j * kThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & mask], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile: keys are taken in index order (iteration j
// covers indices base + j*256 .. +255, warp-major), each key's rank among
// the tile's earlier keys with the same digit is the running count of that
// digit plus the counts of earlier warps plus the rank inside its warp.
__global__ void k_digit_scatter(const uint64_t *keys, const uint32_t *vals, int64_t n,
                                int shift, int nbits, const uint64_t *offs, int ntiles,
                                uint64_t *okeys, uint32_t *ovals)
{
    constexpr int kWarps = kThreads / 32;
    __shared__ uint32_t run[kRadix];
    __shared__ uint32_t wcnt[kWarps][kRadix];
    __shared__ uint64_t goff[kRadix];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    run[threadIdx.x] = 0;
    goff[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * kTile;
    const uint64_t mask = (1ull << nbits) - 1;
    for (int j = 0; j < kItems; ++j) {
        for (int w = 0; w < kWarps; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t i = base + (int64_t)j * kThreads + threadIdx.x;
        const bool ok = i < n;
        const uint64_t key = ok ? keys[i] : 0;
        const uint32_t val = ok ? vals[i] : 0;
        const int d = ok ? (int)((key >> shift) & mask) : kRadix;  // kRadix: none
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (ok && rank == 0) wcnt[wid][d] = __popc(peers);
        __syncthreads();
        // digit-major prefix over warps (thread = digit)
        uint32_t acc = 0;
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = acc;
            acc += c;
        }
        __syncthreads();
        if (ok) {
            const uint64_t pos = goff[d] + run[d] + wcnt[wid][d] + rank;
            okeys[pos] = key;
            ovals[pos] = val;
        }
        __syncthreads();
        run[threadIdx.x] += acc;
        __syncthreads();
    }
}

// ---------------------------------------------------------------- arcs

// Arc keys (tail << b | head) with their lengths: both ways for undirected
// input, one way (second slot unused) for directed input.
__global__ void k_make_arcs(const uint32_t *src, const uint32_t *dst, const uint32_t *w,
                            int64_t m, int64_t n, int b, uint64_t *keys, uint32_t *vals,
                            uint64_t *flags, int *err, int both)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t u = src[e], v = dst[e];
        const uint32_t ww = w ? w[e] : 1u;
        if ((int64_t)u >= n || (int64_t)v >= n) atomicExch(err, CC_ERR_GRAPH);
        if (ww == 0) atomicExch(err, CC_ERR_ARG);
        const uint64_t keep = u != v && (int64_t)u < n && (int64_t)v < n;
        keys[2 * e] = (u << b) | v;
        keys[2 * e + 1] = (v << b) | u;
        vals[2 * e] = ww;
        vals[2 * e + 1] = ww;
        flags[2 * e] = keep;
        flags[2 * e + 1] = both ? keep : 0;
    }
}

__global__ void k_compact(const uint64_t *keys, const uint32_t *vals, const uint64_t *flags,
                          const uint64_t *pos, int64_t n, uint64_t *okeys, uint32_t *ovals)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (flags[i]) {
            okeys[pos[i]] = keys[i];
            ovals[pos[i]] = vals[i];
        }
}

// flags[i] = 1 for the first arc of each run of equal keys; mins[run start]
// = the smallest length of the run.
__global__ void k_first_of_run(const uint64_t *keys, int64_t n, uint64_t *flags)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_run_min(const uint64_t *keys, uint32_t *vals, const uint64_t *flags,
                          int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!flags[i]) continue;
        uint32_t mn = vals[i];
        for (int64_t j = i + 1; j < n && keys[j] == keys[i]; ++j) mn = min(mn, vals[j]);
        vals[i] = mn;
    }
}

// Row offsets from keys sorted by tail: rp[u] = first arc with tail >= u.
__global__ void k_row_ptr(const uint64_t *keys, int64_t a, int64_t n, int b, int64_t *rp)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= a;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cur = i < a ? (int64_t)(keys[i] >> b) : n;
        const int64_t prev = i > 0 ? (int64_t)(keys[i - 1] >> b) : -1;
        for (int64_t u = prev + 1; u <= cur; ++u) rp[u] = i;
    }
}

__global__ void k_heads(const uint64_t *keys, int64_t a, int b, int32_t *col)
{
    const uint64_t mask = (1ull << b) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a;
         i += (int64_t)gridDim.x * blockDim.x)
        col[i] = (int32_t)(keys[i] & mask);
}

// ---------------------------------------------------------------- components

__device__ __forceinline__ int32_t find_root(int32_t *parent, int32_t x)
{
    int32_t p = parent[x];
    while (p != x) {
        const int32_t g = parent[p];
        if (g != p) parent[x] = g;  // path halving (benign race)
        x = p;
        p = g;
    }
    return x;
}

__global__ void k_iota32(int32_t *p, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}

// Union of the endpoints of every arc u -> v with u < v.
// A warp per node, a lane per arc (hub rows no longer run on one thread).
__global__ void k_hook(const int64_t *rp, const int32_t *col, int64_t n, int32_t *parent)
{
    const int lane = threadIdx.x & 31;
    for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < n;
         u += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        for (int64_t e = rp[u] + lane; e < rp[u + 1]; e += 32) {
            const int32_t v = col[e];
            if (v <= u) continue;
            int32_t a = find_root(parent, (int32_t)u), b = find_root(parent, v);
            while (a != b) {
                if (a < b) { const int32_t t = a; a = b; b = t; }  // hook larger under smaller
                const int32_t old = atomicCAS(&parent[a], a, b);
                if (old == a) break;
                a = find_root(parent, old);
                b = find_root(parent, b);
            }
        }
    }
}

// Component label = root, found with reads only (a concurrent path-halving
// write could otherwise replace a freshly written root by a non-root
// ancestor).
__global__ void k_label_count(const int32_t *parent, int64_t n, int32_t *label,
                              uint32_t *size)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t r = (int32_t)v;
        while (parent[r] != r) r = parent[r];
        label[v] = r;
        atomicAdd(&size[r], 1u);
    }
}

// best = max over roots of (size << 32 | ~root): largest, ties to smallest id
__global__ void k_pick(const uint32_t *size, int64_t n, unsigned long long *best)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        if (size[v])
            atomicMax(best, ((unsigned long long)size[v] << 32) |
                                (0xFFFFFFFFull - (unsigned long long)v));
}

__global__ void k_keep_flags(const int32_t *parent, int64_t n, int32_t root, uint64_t *flags)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        flags[v] = parent[v] == root ? 1 : 0;
}

// Degrees of kept nodes (for the new row offsets) and the new id map.
__global__ void k_kept_deg(const int64_t *rp, const uint64_t *flags, const uint64_t *pos,
                           int64_t n, uint64_t *deg, int32_t *newid, int32_t *old_id)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (flags[v]) {
            deg[pos[v]] = (uint64_t)(rp[v + 1] - rp[v]);
            newid[v] = (int32_t)pos[v];
            old_id[pos[v]] = (int32_t)v;
        } else {
            newid[v] = -1;
        }
    }
}

// A neighbour outside the kept component cannot occur for a correct
// labelling; it is reported rather than written.
__global__ void k_rewrite_rows(const int64_t *rp, const int32_t *col, const uint32_t *w,
                               const int32_t *old_id, const int32_t *newid,
                               const uint64_t *nrp, int64_t nk, int32_t *ncol, uint32_t *nw,
                               int *err)
{
    const int lane = threadIdx.x & 31;
    for (int64_t x = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; x < nk;
         x += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t v = old_id[x];
        const int64_t b = rp[v], o = (int64_t)nrp[x];
        for (int64_t e = b + lane; e < rp[v + 1]; e += 32) {
            const int32_t y = newid[col[e]];
            if (y < 0) atomicExch(err, CC_ERR_GRAPH);
            ncol[o + (e - b)] = y < 0 ? 0 : y;
            if (w) nw[o + (e - b)] = w[e];
        }
    }
}

// ---------------------------------------------------------------- directed

// Reverse arc keys (head << b | tail) with the lengths.
__global__ void k_swap_keys(const uint64_t *keys, const uint32_t *vals, int64_t a, int b,
                            uint64_t *okeys, uint32_t *ovals)
{
    const uint64_t mask = (1ull << b) - 1;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t u = keys[e] >> b, v = keys[e] & mask;
        okeys[e] = (v << b) | u;
        ovals[e] = vals[e];
    }
}

// ------------------------------------------------- strongly connected parts
//
// Largest strongly connected component (round trips need strong
// connectivity, section 6.1), found on the device.  Every live node
// carries the label of the part of the graph it lies in; a part holds every
// strongly connected component it meets.  The parts start as the weakly
// connected components.  Each round:
//   trim    a node without an arc from, or without one to, a live node of
//           its own part is a component by itself;
//   stats   per part: size, smallest id and a pivot (largest out x in
//           degree, ties to the smallest id);
//   prune   a part that cannot hold a component beating the best one found
//           so far (fewer nodes, or as many with a larger smallest id) dies;
//   search  forward and backward searches from every pivot, confined to its
//           part; the nodes reached both ways are the pivot's component, the
//           rest of the part splits into three new parts (reached forward
//           only, backward only, neither), each holding whole components.
// Labels: 2n + root for the weak components, p and n + p for the forward-
// and backward-only remainders of pivot p (p never pivots again), the
// remainder reached by neither keeps its label.
constexpr uint64_t kDeadLab = ~0ull;
constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned long long best_key(unsigned size, uint32_t min_id)
{
    return ((unsigned long long)size << 32) | (0xFFFFFFFFull - min_id);
}

__global__ void k_scc_init(const int32_t *parent, int64_t n, uint64_t *lab, int32_t *comp)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        int32_t r = (int32_t)v;
        while (parent[r] != r) r = parent[r];
        lab[v] = (uint64_t)(2 * n + r);
        comp[v] = -1;
    }
}

// True when some arc of row v (a warp scans it 32 arcs at a time) leads to
// a node labelled L.
__device__ __forceinline__ bool row_meets(const int64_t *rp, const int32_t *col,
                                          const uint64_t *lab, int64_t v, uint64_t L, int lane)
{
    const int64_t end = rp[v + 1];
    for (int64_t e0 = rp[v]; e0 < end; e0 += 32) {
        const int64_t e = e0 + lane;
        const bool hit = e < end && lab[col[e]] == L;
        if (__any_sync(kFull, hit)) return true;
    }
    return false;
}

// Trim, a warp per node.  Labels change in place while other warps read
// them: a node seen live or dead either way keeps the decision valid, since
// a trimmed node is a component of its own.
__global__ void k_scc_trim(const int64_t *rp, const int32_t *col, const int64_t *rrp,
                           const int32_t *rcol, int64_t n, uint64_t *lab, int32_t *comp,
                           unsigned long long *removed, unsigned long long *best)
{
    const int lane = threadIdx.x & 31;
    unsigned long long cnt = 0, bk = 0;
    for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < n;
         v += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const uint64_t L = lab[v];
        if (L == kDeadLab) continue;
        if (row_meets(rp, col, lab, v, L, lane) && row_meets(rrp, rcol, lab, v, L, lane))
            continue;
        if (lane == 0) {
            lab[v] = kDeadLab;
            comp[v] = (int32_t)v;
            ++cnt;
            bk = max(bk, best_key(1u, (uint32_t)v));
        }
    }
    if (lane == 0 && cnt) {
        atomicAdd(removed, cnt);
        atomicMax(best, bk);
    }
}

// Per part: size, smallest id, pivot key (out x in degree << 32 | ~id).
// Warps whose live lanes share one part reduce first (the common case: one
// large part).
__global__ void k_scc_stats(const int64_t *rp, const int64_t *rrp, int64_t n,
                            const uint64_t *lab, unsigned long long *pk, unsigned *sz,
                            unsigned *mn)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride) {
        const int64_t v = base + lane;
        const uint64_t L = v < n ? lab[v] : kDeadLab;
        const bool live = L != kDeadLab;
        const unsigned bal = __ballot_sync(kFull, live);
        if (!bal) continue;
        unsigned long long key = 0;
        if (live) {
            const unsigned long long s = (unsigned long long)(rp[v + 1] - rp[v]) *
                                         (unsigned long long)(rrp[v + 1] - rrp[v]);
            key = (min(s, 0xFFFFFFFFull) << 32) | (0xFFFFFFFFull - (uint64_t)v);
        }
        const uint64_t L0 = __shfl_sync(kFull, L, __ffs(bal) - 1);
        if (__all_sync(kFull, !live || L == L0)) {
            unsigned long long k = key;
            unsigned m = live ? (unsigned)v : kFull;
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                k = max(k, __shfl_xor_sync(kFull, k, o));
                m = min(m, __shfl_xor_sync(kFull, m, o));
            }
            if (lane == 0) {
                atomicMax(&pk[L0], k);
                atomicAdd(&sz[L0], (unsigned)__popc(bal));
                atomicMin(&mn[L0], m);
            }
        } else if (live) {
            atomicMax(&pk[L], key);
            atomicAdd(&sz[L], 1u);
            atomicMin(&mn[L], (unsigned)v);
        }
    }
}

// Prune parts that cannot beat the best component so far; queue the pivots
// of the others (both searches start from them).
__global__ void k_scc_seed(int64_t n, uint64_t *lab, const unsigned long long *pk,
                           const unsigned *sz, const unsigned *mn,
                           const unsigned long long *best, unsigned *fw, unsigned *bw,
                           int32_t *q, unsigned long long *qn)
{
    const unsigned long long b = *best;
    const unsigned bs = (unsigned)(b >> 32);
    const unsigned bm = (unsigned)(0xFFFFFFFFull - (b & 0xFFFFFFFFull));
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t L = lab[v];
        if (L == kDeadLab) continue;
        if (sz[L] < bs || (sz[L] == bs && mn[L] > bm)) {
            lab[v] = kDeadLab;
            continue;
        }
        if ((uint32_t)pk[L] == (uint32_t)(0xFFFFFFFFull - (uint64_t)v)) {
            fw[v] = 1u;
            bw[v] = 1u;
            q[atomicAdd(qn, 1ull)] = (int32_t)v;
        }
    }
}

// One level of the confined searches: a warp per queued node, a lane per
// arc; the first to reach a node of the same part queues it (one queue
// reservation per warp step).
__global__ void k_scc_bfs(const int64_t *rp, const int32_t *col, const uint64_t *lab,
                          const int32_t *qin, int64_t nin, int32_t *qout,
                          unsigned long long *nout, unsigned *vis)
{
    const int lane = threadIdx.x & 31;
    for (int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; t < nin;
         t += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t u = qin[t];
        const uint64_t L = lab[u];
        const int64_t end = rp[u + 1];
        for (int64_t e0 = rp[u]; e0 < end; e0 += 32) {
            const int64_t e = e0 + lane;
            int32_t x = -1;
            bool push = false;
            if (e < end) {
                x = col[e];
                push = lab[x] == L && vis[x] == 0u && atomicExch(&vis[x], 1u) == 0u;
            }
            const unsigned bal = __ballot_sync(kFull, push);
            if (!bal) continue;
            unsigned long long at = 0;
            if (lane == __ffs(bal) - 1) at = atomicAdd(nout, (unsigned long long)__popc(bal));
            at = __shfl_sync(kFull, at, __ffs(bal) - 1);
            if (push) qout[at + __popc(bal & ((1u << lane) - 1u))] = x;
        }
    }
}

// Split every searched part: both ways -> the pivot's component (dead),
// forward only -> label p, backward only -> n + p, neither -> unchanged.
__global__ void k_scc_split(int64_t n, uint64_t *lab, const unsigned long long *pk,
                            unsigned *fw, unsigned *bw, int32_t *comp, unsigned *csz,
                            unsigned *cmn)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride) {
        const int64_t v = base + lane;
        const uint64_t L = v < n ? lab[v] : kDeadLab;
        bool in_s = false;
        uint32_t p = 0;
        if (L != kDeadLab) {
            p = (uint32_t)(0xFFFFFFFFull - (pk[L] & 0xFFFFFFFFull));
            const bool f = fw[v] != 0u, b = bw[v] != 0u;
            if (f && b) {
                in_s = true;
                comp[v] = (int32_t)p;
                lab[v] = kDeadLab;
            } else if (f) {
                lab[v] = p;
            } else if (b) {
                lab[v] = (uint64_t)n + p;
            }
            if (f) fw[v] = 0u;
            if (b) bw[v] = 0u;
        }
        const unsigned bal = __ballot_sync(kFull, in_s);
        if (!bal) continue;
        const uint32_t p0 = __shfl_sync(kFull, p, __ffs(bal) - 1);
        if (__all_sync(kFull, !in_s || p == p0)) {
            if (lane == __ffs(bal) - 1) {
                atomicAdd(&csz[p0], (unsigned)__popc(bal));
                atomicMin(&cmn[p0], (unsigned)v);  // lowest member lane: smallest id
            }
        } else if (in_s) {
            atomicAdd(&csz[p], 1u);
            atomicMin(&cmn[p], (unsigned)v);
        }
    }
}

__global__ void k_scc_best(int64_t n, const unsigned *csz, const unsigned *cmn,
                           unsigned long long *best)
{
    unsigned long long k = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        if (csz[v]) k = max(k, best_key(csz[v], cmn[v]));
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) k = max(k, __shfl_xor_sync(kFull, k, o));
    if ((threadIdx.x & 31) == 0 && k) atomicMax(best, k);
}

__global__ void k_comp_flags(const int32_t *comp, int64_t n, int32_t c, uint64_t *flags)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        flags[v] = comp[v] == c ? 1 : 0;
}

// Kept nodes: new ids, and per kept row the arcs whose head is kept too (a
// warp per row).
__global__ void k_kept_arcs(const int64_t *rp, const int32_t *col, const uint64_t *flags,
                            const uint64_t *pos, int64_t n, uint64_t *deg, int32_t *newid,
                            int32_t *old_id)
{
    const int lane = threadIdx.x & 31;
    for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < n;
         v += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        if (!flags[v]) {
            if (lane == 0) newid[v] = -1;
            continue;
        }
        unsigned c = 0;
        for (int64_t e = rp[v] + lane; e < rp[v + 1]; e += 32) c += flags[col[e]] ? 1u : 0u;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        if (lane == 0) {
            deg[pos[v]] = c;
            newid[v] = (int32_t)pos[v];
            old_id[pos[v]] = (int32_t)v;
        }
    }
}

// Kept rows with their kept arcs, in order (ballot compaction per 32 arcs).
__global__ void k_rewrite_kept(const int64_t *rp, const int32_t *col, const uint32_t *w,
                               const uint64_t *flags, const int32_t *old_id,
                               const int32_t *newid, const uint64_t *nrp, int64_t nk,
                               int32_t *ncol, uint32_t *nw)
{
    const int lane = threadIdx.x & 31;
    for (int64_t x = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; x < nk;
         x += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t v = old_id[x];
        int64_t o = (int64_t)nrp[x];
        for (int64_t e0 = rp[v]; e0 < rp[v + 1]; e0 += 32) {
            const int64_t e = e0 + lane;
            const bool in = e < rp[v + 1];
            const int32_t u = in ? col[e] : 0;
            const bool keep = in && flags[u];
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
            if (keep) {
                const int64_t q = o + __popc(bal & ((1u << lane) - 1u));
                ncol[q] = newid[u];
                if (w) nw[q] = w[e];
            }
            o += __popc(bal);
        }
    }
}

__global__ void k_u64_to_i64(const uint64_t *in, int64_t n, int64_t *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int64_t)in[i];
}

__global__ void k_widen(const uint32_t *in, int64_t n, uint64_t *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i];
}

int gsz(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>(1, (n + 255) / 256), 152 * 32); }

struct Buf {
    void *p = nullptr;
    ~Buf() { if (p) cudaFree(p); }
    template <class T> T *as() { return static_cast<T *>(p); }
    int alloc(size_t bytes)
    {
        if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return CC_ERR_OOM;
        }
        return CC_OK;
    }
};

#define G_RC(x)                      \
    do {                             \
        int r_ = (x);                \
        if (r_ != CC_OK) return r_;  \
    } while (0)
#define G_CK(x)                                          \
    do {                                                 \
        const cudaError_t e_ = (x);                      \
        if (e_ != cudaSuccess) {                         \
            note_cuda_error(e_, __FILE__, __LINE__);     \
            cudaGetLastError();                          \
            return CC_ERR_CUDA;                          \
        }                                                \
    } while (0)

// Exclusive scan of n uint64 values (in -> out, may alias), returns the total.
int scan_u64(const uint64_t *in, uint64_t *out, int64_t n, uint64_t *total, cudaStream_t st)
{
    const int per = kThreads * 4;
    const int64_t nb = (n + per - 1) / per;
    Buf sums, offs;
    G_RC(sums.alloc((size_t)std::max<int64_t>(nb, 1) * 8));
    G_RC(offs.alloc((size_t)std::max<int64_t>(nb, 1) * 8));
    if (n > 0) k_tile_sums<<<(int)nb, kThreads, 0, st>>>(in, n, sums.as<uint64_t>());
    uint64_t tot = 0;
    if (nb <= 1) {
        G_CK(cudaMemsetAsync(offs.p, 0, 8, st));
        if (n > 0) G_CK(cudaMemcpyAsync(&tot, sums.p, 8, cudaMemcpyDeviceToHost, st));
    } else {
        G_RC(scan_u64(sums.as<uint64_t>(), offs.as<uint64_t>(), nb, &tot, st));
    }
    if (n > 0) k_tile_scan<<<(int)nb, kThreads, 0, st>>>(in, n, offs.as<uint64_t>(), out);
    G_CK(cudaStreamSynchronize(st));
    *total = tot;
    return CC_OK;
}

// Stable LSD radix sort of (keys, vals) over the low `bits` bits.
int radix_sort(uint64_t *keys, uint32_t *vals, int64_t n, int bits, uint64_t *tk,
               uint32_t *tv, cudaStream_t st, bool *in_tmp)
{
    const int ntiles = (int)((n + kTile - 1) / kTile);
    Buf counts, offs;
    G_RC(counts.alloc((size_t)kRadix * ntiles * 4));
    G_RC(offs.alloc((size_t)kRadix * ntiles * 8));
    Buf c64;
    G_RC(c64.alloc((size_t)kRadix * ntiles * 8));
    uint64_t *ka = keys, *kb = tk;
    uint32_t *va = vals, *vb = tv;
    for (int shift = 0; shift < bits; shift += 8) {
        const int nb = std::min(8, bits - shift);
        k_digit_hist<<<ntiles, kThreads, 0, st>>>(ka, n, shift, nb, counts.as<uint32_t>(),
                                                  ntiles);
        // widen to 64-bit for the scan
        const int64_t nc = (int64_t)kRadix * ntiles;
        k_widen<<<gsz(nc), 256, 0, st>>>(counts.as<uint32_t>(), nc, c64.as<uint64_t>());
        uint64_t tot = 0;
        G_RC(scan_u64(c64.as<uint64_t>(), offs.as<uint64_t>(), nc, &tot, st));
        k_digit_scatter<<<ntiles, kThreads, 0, st>>>(ka, va, n, shift, nb,
                                                     offs.as<uint64_t>(), ntiles, kb, vb);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    G_CK(cudaStreamSynchronize(st));
    *in_tmp = ka != keys;
    return CC_OK;
}


}  // namespace

int device_scan_u64(const uint64_t *in, uint64_t *out, int64_t n, uint64_t *total,
                    cudaStream_t st)
{
    return scan_u64(in, out, n, total, st);
}

int device_radix_sort(uint64_t *keys, uint32_t *vals, int64_t n, int bits, uint64_t *tk,
                      uint32_t *tv, cudaStream_t st, bool *in_tmp)
{
    return radix_sort(keys, vals, n, bits, tk, tv, st, in_tmp);
}

// Undirected graph to CSR on the device (see the top of this file).  On
// success the device buffers rp / col / w (w only when lengths are given)
// are owned by the caller (cudaFree), rp_host and old_id hold host copies.
int build_csr_device(int64_t n, int64_t m, const uint32_t *h_src, const uint32_t *h_dst,
                     const uint32_t *h_w, bool keep_component, DeviceCSR &out)
{
    if (n < 2 || m < 0 || (m > 0 && (!h_src || !h_dst))) return CC_ERR_ARG;
    if (n > 0x7FFFFFFFLL || 2 * m > 0x7FFFFFFFLL) return CC_ERR_TOO_LARGE;
    cudaStream_t st = 0;
    int b = 1;
    while ((1ll << b) < n) ++b;
    const int64_t A0 = 2 * m;
    Buf dsrc, ddst, dw, k0, v0, k1, v1, fl, pos, err;
    G_RC(dsrc.alloc(m * 4));
    G_RC(ddst.alloc(m * 4));
    if (h_w) G_RC(dw.alloc(m * 4));
    G_RC(k0.alloc(A0 * 8));
    G_RC(v0.alloc(A0 * 4));
    G_RC(k1.alloc(A0 * 8));
    G_RC(v1.alloc(A0 * 4));
    const int64_t F = std::max<int64_t>(A0, n) + 1;  // flags over arcs or nodes
    G_RC(fl.alloc(F * 8));
    G_RC(pos.alloc(F * 8));
    G_RC(err.alloc(4));
    if (m > 0) {
        G_CK(cudaMemcpy(dsrc.p, h_src, m * 4, cudaMemcpyHostToDevice));
        G_CK(cudaMemcpy(ddst.p, h_dst, m * 4, cudaMemcpyHostToDevice));
        if (h_w) G_CK(cudaMemcpy(dw.p, h_w, m * 4, cudaMemcpyHostToDevice));
    }
    G_CK(cudaMemset(err.p, 0, 4));
    // 1. arcs both ways, self-loops dropped
    if (m > 0)
        k_make_arcs<<<gsz(m), 256, 0, st>>>(dsrc.as<uint32_t>(), ddst.as<uint32_t>(),
                                            h_w ? dw.as<uint32_t>() : nullptr, m, n, b,
                                            k0.as<uint64_t>(), v0.as<uint32_t>(),
                                            fl.as<uint64_t>(), err.as<int>(), 1);
    int herr = 0;
    G_CK(cudaMemcpy(&herr, err.p, 4, cudaMemcpyDeviceToHost));
    if (herr) return herr;
    uint64_t A1 = 0;
    G_RC(scan_u64(fl.as<uint64_t>(), pos.as<uint64_t>(), A0, &A1, st));
    if (A0 > 0)
        k_compact<<<gsz(A0), 256, 0, st>>>(k0.as<uint64_t>(), v0.as<uint32_t>(),
                                           fl.as<uint64_t>(), pos.as<uint64_t>(), A0,
                                           k1.as<uint64_t>(), v1.as<uint32_t>());
    // 2. sort by (tail, head)
    bool in_tmp = false;
    if (A1 > 0)
        G_RC(radix_sort(k1.as<uint64_t>(), v1.as<uint32_t>(), (int64_t)A1, 2 * b,
                        k0.as<uint64_t>(), v0.as<uint32_t>(), st, &in_tmp));
    uint64_t *ks = in_tmp ? k0.as<uint64_t>() : k1.as<uint64_t>();
    uint32_t *vs = in_tmp ? v0.as<uint32_t>() : v1.as<uint32_t>();
    uint64_t *ko = in_tmp ? k1.as<uint64_t>() : k0.as<uint64_t>();
    uint32_t *vo = in_tmp ? v1.as<uint32_t>() : v0.as<uint32_t>();
    // 3. merge parallel arcs (smallest length)
    uint64_t A2 = 0;
    if (A1 > 0) {
        k_first_of_run<<<gsz(A1), 256, 0, st>>>(ks, (int64_t)A1, fl.as<uint64_t>());
        k_run_min<<<gsz(A1), 256, 0, st>>>(ks, vs, fl.as<uint64_t>(), (int64_t)A1);
        G_RC(scan_u64(fl.as<uint64_t>(), pos.as<uint64_t>(), (int64_t)A1, &A2, st));
        k_compact<<<gsz(A1), 256, 0, st>>>(ks, vs, fl.as<uint64_t>(), pos.as<uint64_t>(),
                                           (int64_t)A1, ko, vo);
    }
    // 4. CSR of all n nodes
    Buf rp, col;
    G_RC(rp.alloc((n + 1) * 8));
    G_RC(col.alloc(std::max<uint64_t>(A2, 1) * 4));
    k_row_ptr<<<gsz((int64_t)A2 + 1), 256, 0, st>>>(ko, (int64_t)A2, n, b, rp.as<int64_t>());
    if (A2 > 0) k_heads<<<gsz(A2), 256, 0, st>>>(ko, (int64_t)A2, b, col.as<int32_t>());
    uint32_t *wv = vo;  // merged lengths, in arc order
    int64_t nk = n;
    Buf nrp, ncol, nw, parent, label, size, newid, oldid, degs, best;
    int64_t *frp = rp.as<int64_t>();
    int32_t *fcol = col.as<int32_t>();
    uint32_t *fw = h_w ? wv : nullptr;
    if (keep_component) {
        // 5. components
        G_RC(parent.alloc(n * 4));
        G_RC(size.alloc(n * 4));
        G_RC(best.alloc(8));
        G_CK(cudaMemset(size.p, 0, n * 4));
        G_CK(cudaMemset(best.p, 0, 8));
        k_iota32<<<gsz(n), 256, 0, st>>>(parent.as<int32_t>(), n);
        k_hook<<<gsz(n * 32), 256, 0, st>>>(frp, fcol, n, parent.as<int32_t>());
        G_RC(label.alloc(n * 4));
        k_label_count<<<gsz(n), 256, 0, st>>>(parent.as<int32_t>(), n, label.as<int32_t>(),
                                              size.as<uint32_t>());
        k_pick<<<gsz(n), 256, 0, st>>>(size.as<uint32_t>(), n,
                                       best.as<unsigned long long>());
        unsigned long long hb = 0;
        G_CK(cudaMemcpy(&hb, best.p, 8, cudaMemcpyDeviceToHost));
        const int32_t root = (int32_t)(0xFFFFFFFFull - (hb & 0xFFFFFFFFull));
        // 6. renumber the kept nodes and rewrite their rows
        k_keep_flags<<<gsz(n), 256, 0, st>>>(label.as<int32_t>(), n, root, fl.as<uint64_t>());
        uint64_t kept = 0;
        G_RC(scan_u64(fl.as<uint64_t>(), pos.as<uint64_t>(), n, &kept, st));
        nk = (int64_t)kept;
        if (nk < 2) return CC_ERR_GRAPH;
        G_RC(newid.alloc(n * 4));
        G_RC(oldid.alloc(nk * 4));
        G_RC(degs.alloc((nk + 1) * 8));
        k_kept_deg<<<gsz(n), 256, 0, st>>>(frp, fl.as<uint64_t>(), pos.as<uint64_t>(), n,
                                           degs.as<uint64_t>(), newid.as<int32_t>(),
                                           oldid.as<int32_t>());
        uint64_t arcs = 0;
        G_RC(scan_u64(degs.as<uint64_t>(), degs.as<uint64_t>(), nk, &arcs, st));
        G_CK(cudaMemcpy(degs.as<uint64_t>() + nk, &arcs, 8, cudaMemcpyHostToDevice));
        G_RC(nrp.alloc((nk + 1) * 8));
        G_RC(ncol.alloc(std::max<uint64_t>(arcs, 1) * 4));
        if (h_w) G_RC(nw.alloc(std::max<uint64_t>(arcs, 1) * 4));
        k_u64_to_i64<<<gsz(nk + 1), 256, 0, st>>>(degs.as<uint64_t>(), nk + 1,
                                                  nrp.as<int64_t>());
        k_rewrite_rows<<<gsz(nk * 32), 256, 0, st>>>(frp, fcol, fw, oldid.as<int32_t>(),
                                                newid.as<int32_t>(), degs.as<uint64_t>(), nk,
                                                ncol.as<int32_t>(),
                                                h_w ? nw.as<uint32_t>() : nullptr, err.as<int>());
        G_CK(cudaMemcpy(&herr, err.p, 4, cudaMemcpyDeviceToHost));
        if (herr) return herr;
        out.arcs = (int64_t)arcs;
        out.old_id.resize(nk);
        G_CK(cudaMemcpy(out.old_id.data(), oldid.p, nk * 4, cudaMemcpyDeviceToHost));
        std::swap(out.rp, nrp.p);
        std::swap(out.col, ncol.p);
        if (h_w) std::swap(out.w, nw.p);
    } else {
        out.arcs = (int64_t)A2;
        out.old_id.resize(n);
        for (int64_t v = 0; v < n; ++v) out.old_id[v] = (int32_t)v;
        if (h_w) {
            G_RC(nw.alloc(std::max<uint64_t>(A2, 1) * 4));
            if (A2) G_CK(cudaMemcpy(nw.p, wv, A2 * 4, cudaMemcpyDeviceToDevice));
            std::swap(out.w, nw.p);
        }
        std::swap(out.rp, rp.p);
        std::swap(out.col, col.p);
    }
    out.n = nk;
    out.rp_host.resize(nk + 1);
    G_CK(cudaMemcpy(out.rp_host.data(), out.rp, (nk + 1) * 8, cudaMemcpyDeviceToHost));
    G_CK(cudaDeviceSynchronize());
    return CC_OK;
}

// Sorted, merged arcs (keys tail << b | head, lengths) -> CSR over n nodes.
static int csr_from_sorted(const uint64_t *keys, const uint32_t *vals, int64_t a, int64_t n, int b,
                           bool weighted, Buf &rp, Buf &col, Buf &w, cudaStream_t st)
{
    G_RC(rp.alloc((n + 1) * 8));
    G_RC(col.alloc(std::max<int64_t>(a, 1) * 4));
    k_row_ptr<<<gsz(a + 1), 256, 0, st>>>(keys, a, n, b, rp.as<int64_t>());
    if (a > 0) k_heads<<<gsz(a), 256, 0, st>>>(keys, a, b, col.as<int32_t>());
    if (weighted) {
        G_RC(w.alloc(std::max<int64_t>(a, 1) * 4));
        if (a > 0) G_CK(cudaMemcpyAsync(w.p, vals, a * 4, cudaMemcpyDeviceToDevice, st));
    }
    return CC_OK;
}

// Rows of the kept nodes with their kept arcs, renumbered.
static int filter_csr(const int64_t *rp, const int32_t *col, const uint32_t *w, int64_t n,
                      const uint64_t *flags, const uint64_t *pos, int64_t nk, Buf &newid,
                      Buf &oldid, DeviceCSR &out, cudaStream_t st)
{
    Buf degs, nrp, ncol, nw;
    G_RC(degs.alloc((nk + 1) * 8));
    k_kept_arcs<<<gsz(n * 32), 256, 0, st>>>(rp, col, flags, pos, n, degs.as<uint64_t>(),
                                             newid.as<int32_t>(), oldid.as<int32_t>());
    uint64_t arcs = 0;
    G_RC(scan_u64(degs.as<uint64_t>(), degs.as<uint64_t>(), nk, &arcs, st));
    G_CK(cudaMemcpy(degs.as<uint64_t>() + nk, &arcs, 8, cudaMemcpyHostToDevice));
    G_RC(nrp.alloc((nk + 1) * 8));
    G_RC(ncol.alloc(std::max<uint64_t>(arcs, 1) * 4));
    if (w) G_RC(nw.alloc(std::max<uint64_t>(arcs, 1) * 4));
    k_u64_to_i64<<<gsz(nk + 1), 256, 0, st>>>(degs.as<uint64_t>(), nk + 1, nrp.as<int64_t>());
    k_rewrite_kept<<<gsz(nk * 32), 256, 0, st>>>(rp, col, w, flags, oldid.as<int32_t>(),
                                                 newid.as<int32_t>(), degs.as<uint64_t>(), nk,
                                                 ncol.as<int32_t>(), w ? nw.as<uint32_t>() : nullptr);
    out.n = nk;
    out.arcs = (int64_t)arcs;
    std::swap(out.rp, nrp.p);
    std::swap(out.col, ncol.p);
    if (w) std::swap(out.w, nw.p);
    out.rp_host.resize(nk + 1);
    G_CK(cudaMemcpy(out.rp_host.data(), out.rp, (nk + 1) * 8, cudaMemcpyDeviceToHost));
    return CC_OK;
}

// Largest strongly connected component (see the kernels above): flags[v] =
// 1 for its nodes, *kept = its size.  Ties go to the component holding the
// smallest id.
static int largest_scc(const int64_t *rp, const int32_t *col, const int64_t *rrp,
                       const int32_t *rcol, int64_t n, uint64_t *flags, int64_t *kept,
                       cudaStream_t st)
{
    Buf parent, lab, comp, fw, bw, qp, q0, q1, pk, sz, mn, csz, cmn, ctr;
    const int64_t nl = 3 * n;  // label space
    G_RC(parent.alloc(n * 4));
    G_RC(lab.alloc(n * 8));
    G_RC(comp.alloc(n * 4));
    G_RC(fw.alloc(n * 4));
    G_RC(bw.alloc(n * 4));
    G_RC(qp.alloc(n * 4));
    G_RC(q0.alloc(n * 4));
    G_RC(q1.alloc(n * 4));
    G_RC(pk.alloc(nl * 8));
    G_RC(sz.alloc(nl * 4));
    G_RC(mn.alloc(nl * 4));
    G_RC(csz.alloc(n * 4));
    G_RC(cmn.alloc(n * 4));
    G_RC(ctr.alloc(3 * 8));  // best, removed, queue count
    unsigned long long *best = ctr.as<unsigned long long>(), *removed = best + 1,
                       *qn = best + 2;
    // weak components by union-find over the arcs of G and of G^T
    k_iota32<<<gsz(n), 256, 0, st>>>(parent.as<int32_t>(), n);
    k_hook<<<gsz(n * 32), 256, 0, st>>>(rp, col, n, parent.as<int32_t>());
    k_hook<<<gsz(n * 32), 256, 0, st>>>(rrp, rcol, n, parent.as<int32_t>());
    k_scc_init<<<gsz(n), 256, 0, st>>>(parent.as<int32_t>(), n, lab.as<uint64_t>(),
                                       comp.as<int32_t>());
    G_CK(cudaMemsetAsync(fw.p, 0, n * 4, st));
    G_CK(cudaMemsetAsync(bw.p, 0, n * 4, st));
    G_CK(cudaMemsetAsync(csz.p, 0, n * 4, st));
    G_CK(cudaMemsetAsync(cmn.p, 0xFF, n * 4, st));
    G_CK(cudaMemsetAsync(best, 0, 8, st));
    uint64_t *L = lab.as<uint64_t>();
    for (;;) {
        // trim while it removes nodes (at most 16 sweeps a round; the
        // searches settle whatever is left)
        for (int it = 0; it < 16; ++it) {
            G_CK(cudaMemsetAsync(removed, 0, 8, st));
            k_scc_trim<<<gsz(n * 32), 256, 0, st>>>(rp, col, rrp, rcol, n, L,
                                                    comp.as<int32_t>(), removed, best);
            unsigned long long h = 0;
            G_CK(cudaMemcpyAsync(&h, removed, 8, cudaMemcpyDeviceToHost, st));
            G_CK(cudaStreamSynchronize(st));
            if (h == 0) break;
        }
        G_CK(cudaMemsetAsync(pk.p, 0, nl * 8, st));
        G_CK(cudaMemsetAsync(sz.p, 0, nl * 4, st));
        G_CK(cudaMemsetAsync(mn.p, 0xFF, nl * 4, st));
        G_CK(cudaMemsetAsync(qn, 0, 8, st));
        k_scc_stats<<<gsz(n), 256, 0, st>>>(rp, rrp, n, L, pk.as<unsigned long long>(),
                                            sz.as<unsigned>(), mn.as<unsigned>());
        k_scc_seed<<<gsz(n), 256, 0, st>>>(n, L, pk.as<unsigned long long>(), sz.as<unsigned>(),
                                           mn.as<unsigned>(), best, fw.as<unsigned>(),
                                           bw.as<unsigned>(), qp.as<int32_t>(), qn);
        unsigned long long npiv = 0;
        G_CK(cudaMemcpyAsync(&npiv, qn, 8, cudaMemcpyDeviceToHost, st));
        G_CK(cudaStreamSynchronize(st));
        if (npiv == 0) break;  // every part settled or pruned
        for (int dir = 0; dir < 2; ++dir) {
            const int64_t *r = dir ? rrp : rp;
            const int32_t *c = dir ? rcol : col;
            unsigned *vis = dir ? bw.as<unsigned>() : fw.as<unsigned>();
            int32_t *qin = q0.as<int32_t>(), *qout = q1.as<int32_t>();
            G_CK(cudaMemcpyAsync(qin, qp.p, npiv * 4, cudaMemcpyDeviceToDevice, st));
            int64_t nin = (int64_t)npiv;
            while (nin > 0) {
                G_CK(cudaMemsetAsync(qn, 0, 8, st));
                k_scc_bfs<<<gsz(nin * 32), 256, 0, st>>>(r, c, L, qin, nin, qout, qn, vis);
                unsigned long long h = 0;
                G_CK(cudaMemcpyAsync(&h, qn, 8, cudaMemcpyDeviceToHost, st));
                G_CK(cudaStreamSynchronize(st));
                nin = (int64_t)h;
                std::swap(qin, qout);
            }
        }
        k_scc_split<<<gsz(n), 256, 0, st>>>(n, L, pk.as<unsigned long long>(), fw.as<unsigned>(),
                                            bw.as<unsigned>(), comp.as<int32_t>(),
                                            csz.as<unsigned>(), cmn.as<unsigned>());
        k_scc_best<<<gsz(n), 256, 0, st>>>(n, csz.as<unsigned>(), cmn.as<unsigned>(), best);
    }
    unsigned long long hb = 0;
    G_CK(cudaMemcpyAsync(&hb, best, 8, cudaMemcpyDeviceToHost, st));
    G_CK(cudaStreamSynchronize(st));
    const int64_t size = (int64_t)(hb >> 32);
    const int64_t min_id = (int64_t)(0xFFFFFFFFull - (hb & 0xFFFFFFFFull));
    if (size < 2 || min_id >= n) {
        *kept = size;
        return CC_OK;
    }
    int32_t c = -1;
    G_CK(cudaMemcpyAsync(&c, comp.as<int32_t>() + min_id, 4, cudaMemcpyDeviceToHost, st));
    G_CK(cudaStreamSynchronize(st));
    k_comp_flags<<<gsz(n), 256, 0, st>>>(comp.as<int32_t>(), n, c, flags);
    *kept = size;
    return CC_OK;
}

int build_csr_device_directed(int64_t n, int64_t m, const uint32_t *h_src, const uint32_t *h_dst,
                              const uint32_t *h_w, bool keep_component, DeviceCSR &F,
                              DeviceCSR &R)
{
    if (n < 2 || m < 0 || (m > 0 && (!h_src || !h_dst))) return CC_ERR_ARG;
    if (n > 0x7FFFFFFFLL || m > 0x7FFFFFFFLL) return CC_ERR_TOO_LARGE;
    cudaStream_t st = 0;
    int b = 1;
    while ((1ll << b) < n) ++b;
    const int64_t A0 = 2 * m;  // k_make_arcs writes two slots per input edge
    Buf dsrc, ddst, dw, k0, v0, k1, v1, fl, pos, err;
    G_RC(dsrc.alloc(m * 4));
    G_RC(ddst.alloc(m * 4));
    if (h_w) G_RC(dw.alloc(m * 4));
    G_RC(k0.alloc(std::max<int64_t>(A0, 1) * 8));
    G_RC(v0.alloc(std::max<int64_t>(A0, 1) * 4));
    G_RC(k1.alloc(std::max<int64_t>(A0, 1) * 8));
    G_RC(v1.alloc(std::max<int64_t>(A0, 1) * 4));
    const int64_t FL = std::max<int64_t>(A0, n) + 1;
    G_RC(fl.alloc(FL * 8));
    G_RC(pos.alloc(FL * 8));
    G_RC(err.alloc(4));
    if (m > 0) {
        G_CK(cudaMemcpy(dsrc.p, h_src, m * 4, cudaMemcpyHostToDevice));
        G_CK(cudaMemcpy(ddst.p, h_dst, m * 4, cudaMemcpyHostToDevice));
        if (h_w) G_CK(cudaMemcpy(dw.p, h_w, m * 4, cudaMemcpyHostToDevice));
    }
    G_CK(cudaMemset(err.p, 0, 4));
    // 1. arcs one way, self-loops dropped; sorted by (tail, head); parallel
    //    arcs merged (smallest length)
    if (m > 0)
        k_make_arcs<<<gsz(m), 256, 0, st>>>(dsrc.as<uint32_t>(), ddst.as<uint32_t>(),
                                            h_w ? dw.as<uint32_t>() : nullptr, m, n, b,
                                            k0.as<uint64_t>(), v0.as<uint32_t>(),
                                            fl.as<uint64_t>(), err.as<int>(), 0);
    int herr = 0;
    G_CK(cudaMemcpy(&herr, err.p, 4, cudaMemcpyDeviceToHost));
    if (herr) return herr;
    uint64_t A1 = 0;
    G_RC(scan_u64(fl.as<uint64_t>(), pos.as<uint64_t>(), A0, &A1, st));
    if (A0 > 0)
        k_compact<<<gsz(A0), 256, 0, st>>>(k0.as<uint64_t>(), v0.as<uint32_t>(),
                                           fl.as<uint64_t>(), pos.as<uint64_t>(), A0,
                                           k1.as<uint64_t>(), v1.as<uint32_t>());
    bool in_tmp = false;
    if (A1 > 0)
        G_RC(radix_sort(k1.as<uint64_t>(), v1.as<uint32_t>(), (int64_t)A1, 2 * b,
                        k0.as<uint64_t>(), v0.as<uint32_t>(), st, &in_tmp));
    uint64_t *ks = in_tmp ? k0.as<uint64_t>() : k1.as<uint64_t>();
    uint32_t *vs = in_tmp ? v0.as<uint32_t>() : v1.as<uint32_t>();
    uint64_t *ko = in_tmp ? k1.as<uint64_t>() : k0.as<uint64_t>();
    uint32_t *vo = in_tmp ? v1.as<uint32_t>() : v0.as<uint32_t>();
    uint64_t A2 = 0;
    if (A1 > 0) {
        k_first_of_run<<<gsz(A1), 256, 0, st>>>(ks, (int64_t)A1, fl.as<uint64_t>());
        k_run_min<<<gsz(A1), 256, 0, st>>>(ks, vs, fl.as<uint64_t>(), (int64_t)A1);
        G_RC(scan_u64(fl.as<uint64_t>(), pos.as<uint64_t>(), (int64_t)A1, &A2, st));
        k_compact<<<gsz(A1), 256, 0, st>>>(ks, vs, fl.as<uint64_t>(), pos.as<uint64_t>(),
                                           (int64_t)A1, ko, vo);
    }
    // 2. forward CSR (G) and reverse CSR (G^T, from the swapped keys)
    Buf frp, fcol, fw, rrp, rcol, rw;
    G_RC(csr_from_sorted(ko, vo, (int64_t)A2, n, b, h_w != nullptr, frp, fcol, fw, st));
    if (A2 > 0) {
        k_swap_keys<<<gsz(A2), 256, 0, st>>>(ko, vo, (int64_t)A2, b, ks, vs);
        G_RC(radix_sort(ks, vs, (int64_t)A2, 2 * b, ko, vo, st, &in_tmp));
    }
    const uint64_t *rks = (A2 > 0 && in_tmp) ? ko : ks;
    const uint32_t *rvs = (A2 > 0 && in_tmp) ? vo : vs;
    G_RC(csr_from_sorted(rks, rvs, (int64_t)A2, n, b, h_w != nullptr, rrp, rcol, rw, st));
    // 3. the largest strongly connected component (largest_scc), unless
    //    every node is kept
    if (!keep_component) {
        std::vector<int32_t> ids(n);
        for (int64_t v = 0; v < n; ++v) ids[v] = (int32_t)v;
        for (DeviceCSR *o : {&F, &R}) {
            o->n = n;
            o->arcs = (int64_t)A2;
            o->old_id = ids;
            o->rp_host.resize(n + 1);
        }
        std::swap(F.rp, frp.p); std::swap(F.col, fcol.p); if (h_w) std::swap(F.w, fw.p);
        std::swap(R.rp, rrp.p); std::swap(R.col, rcol.p); if (h_w) std::swap(R.w, rw.p);
        G_CK(cudaMemcpy(F.rp_host.data(), F.rp, (n + 1) * 8, cudaMemcpyDeviceToHost));
        G_CK(cudaMemcpy(R.rp_host.data(), R.rp, (n + 1) * 8, cudaMemcpyDeviceToHost));
        return CC_OK;
    }
    int64_t nk = 0;
    G_RC(largest_scc(frp.as<int64_t>(), fcol.as<int32_t>(), rrp.as<int64_t>(),
                     rcol.as<int32_t>(), n, fl.as<uint64_t>(), &nk, st));
    if (nk < 2) return CC_ERR_GRAPH;
    uint64_t kept = 0;
    G_RC(scan_u64(fl.as<uint64_t>(), pos.as<uint64_t>(), n, &kept, st));
    if ((int64_t)kept != nk) return CC_ERR_CUDA;  // flags disagree with the component size
    // 4. renumber the kept nodes (increasing original id) and keep the arcs
    //    between them, in G and in G^T
    Buf newid, oldid, newid2, oldid2;
    G_RC(newid.alloc(n * 4));
    G_RC(oldid.alloc(nk * 4));
    G_RC(newid2.alloc(n * 4));
    G_RC(oldid2.alloc(nk * 4));
    G_RC(filter_csr(frp.as<int64_t>(), fcol.as<int32_t>(), h_w ? fw.as<uint32_t>() : nullptr, n,
                    fl.as<uint64_t>(), pos.as<uint64_t>(), nk, newid, oldid, F, st));
    G_RC(filter_csr(rrp.as<int64_t>(), rcol.as<int32_t>(), h_w ? rw.as<uint32_t>() : nullptr, n,
                    fl.as<uint64_t>(), pos.as<uint64_t>(), nk, newid2, oldid2, R, st));
    F.old_id.resize(nk);
    G_CK(cudaMemcpy(F.old_id.data(), oldid.p, nk * 4, cudaMemcpyDeviceToHost));
    R.old_id = F.old_id;
    G_CK(cudaDeviceSynchronize());
    return CC_OK;
}

}  // namespace ccg
