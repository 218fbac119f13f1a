// Device functions of the bit-packed multi-source BFS (see msbfs.cu for the
// method).  A pass runs on a *team* of co-resident CTAs -- the whole grid for
// a single graph, a slice of it when several graphs share one persistent
// launch -- with team-wide barriers on a control block of its own.
#pragma once
#include <cstdint>

#include "barrier.cuh"
#include "cc_internal.h"

namespace ccg {
namespace {


constexpr unsigned FULL = 0xFFFFFFFFu;
// Independent gathers in flight per lane and step: top-down pushes and
// bottom-up scans of light nodes (kUnroll), of medium nodes (kUnrollM) and
// of heavy chunk tasks (kUnrollH); build-time tunables.
#ifndef CC_MSBFS_UNROLL
#define CC_MSBFS_UNROLL 4
#endif
#ifndef CC_MSBFS_UNROLL_M
#define CC_MSBFS_UNROLL_M 4
#endif
#ifndef CC_MSBFS_UNROLL_H
#define CC_MSBFS_UNROLL_H 4
#endif
// Heavy chunk tasks' column indices staged in shared memory by cp.async (1)
// or read from global memory after an L2 prefetch (0).
#ifndef CC_MSBFS_STAGE
#define CC_MSBFS_STAGE 1
#endif
// Shared-memory slots of a warp's staged chunk: entries from b & ~3 (so
// that every 16-byte copy is aligned) up to 3 past its end.
constexpr int kHubSlots = CC_CHUNK + 8;
// Heavy chunk tasks a warp takes from the level's counter at a time.
#ifndef CC_MSBFS_GRAB
#define CC_MSBFS_GRAB 4
#endif
constexpr int kGrab = CC_MSBFS_GRAB;
constexpr int kUnroll = CC_MSBFS_UNROLL;
constexpr int kUnrollM = CC_MSBFS_UNROLL_M;
constexpr int kUnrollH = CC_MSBFS_UNROLL_H;

// Hint: the 128-byte line holding p is read soon; bring it to the L2.
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bits of word w that do not correspond to a source (index >= k): preset in
// visited so that "all bits set" means "reached by every source".
__device__ __forceinline__ uint64_t pad_mask(int k, int w)
{
    const int lo = w * 64;
    if (k <= lo) return ~0ull;
    if (k >= lo + 64) return 0ull;
    return ~0ull << (k - lo);
}

// 32 x 32 bit-matrix transpose across a warp: on return lane c holds, in
// bit r, bit c of the value lane r passed in.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane)
{
#pragma unroll
    for (int j = 16; j >= 1; j >>= 1) {
        const uint32_t m = j == 16 ? 0x0000FFFFu
                         : j == 8  ? 0x00FF00FFu
                         : j == 4  ? 0x0F0F0F0Fu
                         : j == 2  ? 0x33333333u
                                   : 0x55555555u;
        const uint32_t y = __shfl_xor_sync(FULL, x, j);
        x = (lane & j) ? ((x & ~m) | ((y & ~m) >> j))
                       : ((x & m) | ((y & m) << j));
    }
    return x;
}

// Per-lane counts of one level, flushed at its end.  32 bits suffice: a
// lane's share of a level is below the arc count (< 2^31).  They are live
// through the whole pass, so they are kept few and narrow (every register
// here is one less for the scans, and the pass runs at 64 per thread).
struct LaneAcc {
    unsigned ef, eu_dec, words, ninc_dec, nfront;
};

// Update, reduce and enqueue one warp tile.  Lanes form groups of W; group
// g = lane / W is one node (valid or not), lane % W its word.  Must be
// called by all 32 lanes together.
template <int W>
__device__ __forceinline__ void tile_reduce(const BfsJob &J, int l, bool valid,
                                            int v, uint64_t vis, uint64_t nw,
                                            int64_t deg, uint64_t *Fout,
                                            LaneAcc &A, unsigned *s_hist,
                                            bool clear_tflag)
{
    const int lane = threadIdx.x & 31;
    const int w = lane & (W - 1);
    const int64_t vw = (int64_t)v * W + w;
    // Frontier and visited words are written only when new bits arrive.  A
    // frontier word left unwritten keeps bits of an older level of the same
    // parity; each such source reached every neighbour one level after this
    // node, so those bits are already in the neighbours' visited words and
    // are masked off wherever the word is read.
    if (valid && nw) {
        Fout[vw] = nw;
        J.vis[vw] = vis | nw;
    }
    int sx = -1;
    if (valid && (J.red & (RED_DCC | RED_HIST | RED_LC | RED_BAND))) sx = J.sidx[v];
    int c = __popcll(nw);
    int cL = 0;
    unsigned long long xs = 0;
    if ((J.red & RED_LC) && valid && sx < 0 && nw) {
        const uint64_t lm = J.Lmask[vw];
        cL = __popcll(nw & lm);
        if (J.red & RED_SQ) {
            const uint8_t f = J.sqflag[v];
            if (f) {
                const int p = J.pivot[v];
                if (f & 1) {
                    // Sources beyond the threshold reaching v now, at level l.
                    uint64_t bh = nw & ~lm;
                    while (bh) {
                        const int i = w * 64 + __ffsll((long long)bh) - 1;
                        bh &= bh - 1;
                        const long long e = (long long)l - J.dcc[(int64_t)p * J.dcc_k + i];
                        xs += (unsigned long long)(e * e);
                    }
                }
                if (f & 2) {
                    const int is = J.istar[p];
                    if ((is >> 6) == w && ((nw >> (is & 63)) & 1ull)) J.fdist[v] = (uint32_t)l;
                }
            }
        }
    }
    int had = (vis & ~pad_mask(J.k, w)) != 0;
    int done_before = vis == ~0ull;
    int done_after = (vis | nw) == ~0ull;
    int pv = nw ? (w * 64 + __ffsll((long long)nw) - 1) : 0x7FFFFFFF;
#pragma unroll
    for (int o = 1; o < W; o <<= 1) {
        c += __shfl_xor_sync(FULL, c, o);
        cL += __shfl_xor_sync(FULL, cL, o);
        xs += __shfl_xor_sync(FULL, xs, o);
        had |= __shfl_xor_sync(FULL, had, o);
        done_before &= __shfl_xor_sync(FULL, done_before, o);
        done_after &= __shfl_xor_sync(FULL, done_after, o);
        pv = min(pv, __shfl_xor_sync(FULL, pv, o));
    }
    const bool leader = valid && w == 0;
    // (l + 1) eps_a <= eps_b puts every bit of level l in L(v) whatever
    // Delta(v) >= 1: nothing to record (all levels of a small-diameter
    // graph).
    if ((J.red & RED_BAND) && valid && sx < 0 && c > 0 &&
        ((uint64_t)l + 1u) * J.eps_a > J.eps_b) {
        // The hybrid's classification on arrival (section 3's use of the
        // triangle inequality): d(c(v), c_i) lies within l -+ Delta(v).  The
        // class is the same for the W lanes of v (same l and Delta).
        // lc2 collects the complement of L(v) (the sums over HC(v)), so a
        // node whose bits all land in L(v) -- every node of a graph of
        // small diameter -- writes nothing here.
        const uint64_t Dv = had ? (uint64_t)J.delta[v] : (uint64_t)l;
        const uint64_t ul = (uint64_t)l;
        if ((ul - Dv) * J.eps_a > Dv * J.eps_b) {
            if (leader) {  // in HC(v); bflag bit 2: lc2[v] holds sums
                const uint8_t f = J.bflag[v];
                const uint64_t s1 = ul * (uint64_t)c, s2 = ul * ul * (uint64_t)c;
                if (f & 2) {
                    J.lc2[2 * (int64_t)v] += s1;
                    J.lc2[2 * (int64_t)v + 1] += s2;
                } else {
                    J.lc2[2 * (int64_t)v] = s1;
                    J.lc2[2 * (int64_t)v + 1] = s2;
                    J.bflag[v] = f | 2;
                }
            }
        } else if ((ul + Dv) * J.eps_a > Dv * J.eps_b) {
            // Deferred: a byte per source, the first such level clearing
            // the row (each lane its own word's 64 bytes).
            const uint64_t o = ul + Dv - Dv * J.eps_b / J.eps_a;  // 1 .. 2 Delta
            uint8_t *row = J.band + (int64_t)v * (64 * W) + 64 * w;
            const unsigned gmask =
                W == 32 ? FULL : (((1u << (W & 31)) - 1u) << ((lane / W) * W));
            const uint8_t f = J.bflag[v];  // bit 1: v's band row is cleared
            __syncwarp(gmask);               // every lane of v has read it
            if (!(f & 1)) {
                uint4 *r4 = reinterpret_cast<uint4 *>(row);
                const uint4 z = make_uint4(0u, 0u, 0u, 0u);
                r4[0] = z; r4[1] = z; r4[2] = z; r4[3] = z;
                if (leader) J.bflag[v] = f | 1;
            }
            if (o > 255u) {
                if (leader) J.ctl->band_ovf = 1;
            } else {
                uint64_t bb = nw;
                while (bb) {
                    row[__ffsll((long long)bb) - 1] = (uint8_t)o;
                    bb &= bb - 1;
                }
            }
        }
    }
    if (leader && c > 0) {
        const uint64_t ul = (uint64_t)l;
        if (J.red & RED_SUM) {
            J.sum2[2 * (int64_t)v] += ul * (uint64_t)c;
            J.sum2[2 * (int64_t)v + 1] += ul * ul * (uint64_t)c;
        }
        if (cL > 0) {
            J.lc2[2 * (int64_t)v] += ul * (uint64_t)cL;
            J.lc2[2 * (int64_t)v + 1] += ul * ul * (uint64_t)cL;
        }
        if (xs) {
            const uint64_t lo = J.hcse[2 * (int64_t)v] + xs;
            J.hcse[2 * (int64_t)v + 1] += lo < xs ? 1u : 0u;
            J.hcse[2 * (int64_t)v] = lo;
        }
        if ((J.red & RED_PIVOT) && !had) {
            J.pivot[v] = pv;
            J.delta[v] = (uint32_t)l;
        }
    }
    if (leader && clear_tflag) J.tflag[v] = 0u;
    if ((J.red & RED_LEVELS) && valid && nw) {
        uint64_t b = nw;
        while (b) {
            const int i = w * 64 + __ffsll((long long)b) - 1;
            b &= b - 1;
            J.dist_out[(int64_t)v * J.dist_ld + i] = (uint32_t)l;
        }
    }
    if ((J.red & RED_DCC) && sx >= 0 && nw) {
        uint64_t b = nw;
        while (b) {
            const int i = w * 64 + __ffsll((long long)b) - 1;
            b &= b - 1;
            J.dcc[(int64_t)i * J.dcc_k + sx] = (uint32_t)l;
        }
    }
    if (J.red & RED_HIST) {
        const uint64_t x = (valid && sx < 0) ? nw : 0ull;
        if constexpr (W <= 8) {
            if (__ballot_sync(FULL, x != 0ull)) {
                const uint32_t lo = warp_transpose32((uint32_t)x, lane);
                const uint32_t hi = warp_transpose32((uint32_t)(x >> 32), lane);
                constexpr uint32_t M0 = W == 1 ? 0xFFFFFFFFu
                                      : W == 2 ? 0x55555555u
                                      : W == 4 ? 0x11111111u
                                               : 0x01010101u;
#pragma unroll
                for (int s = 0; s < W; ++s) {
                    // lane holds the counts of sources s*64 + lane and
                    // s*64 + 32 + lane (distinct banks: no conflicts)
                    const unsigned c0 = __popc(lo & (M0 << s));
                    const unsigned c1 = __popc(hi & (M0 << s));
                    if (c0) atomicAdd(&s_hist[s * 64 + lane], c0);
                    if (c1) atomicAdd(&s_hist[s * 64 + 32 + lane], c1);
                }
            }
        } else {
            uint64_t b = x;
            while (b) {
                const int i = w * 64 + __ffsll((long long)b) - 1;
                b &= b - 1;
                atomicAdd(&s_hist[i], 1u);
            }
        }
    }
    // Stamp frontier nodes with the level (a later top-down level builds its
    // queue from the stamps) and count level statistics.
    const bool fr = leader && c > 0;
    if (fr) {
        J.fstamp[v] = (uint32_t)l;
        A.ef += (unsigned)deg;
        A.nfront += 1;
    }
    if (leader && done_after && !done_before) {
        A.eu_dec += (unsigned)deg;
        A.ninc_dec += 1;
    }
}

// The words gathered on level l (the pass total and the level's trace).
__device__ __forceinline__ void flush_words(Ctl *ctl, int l, unsigned words)
{
    unsigned long long x = words;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    if ((threadIdx.x & 31) == 0 && x) {
        atomicAdd(&ctl->words, x);
        if (l < kTraceLevels) atomicAdd(&ctl->lvl_words[l], x);
    }
}

// OR of `x` over the lanes holding the same word slot (lane % W).
template <int W>
__device__ __forceinline__ uint64_t or_same_word(uint64_t x)
{
#pragma unroll
    for (int o = W; o < 32; o <<= 1) x |= __shfl_xor_sync(FULL, x, o);
    return x;
}

// OR of the frontier words (slot w) of the columns in c; the U gathers are
// independent, so they are all in flight together.
template <int W, int U>
__device__ __forceinline__ uint64_t gather_cols(const uint64_t *Fin, const int (&c)[U], int w,
                                                unsigned &words)
{
    uint64_t f = 0;
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (c[u] >= 0) {
            f |= Fin[(int64_t)c[u] * W + w];
            words += 1;
        }
    return f;
}

// Column indices row[x], row[x+stride], ... (U of them; -1 from len on),
// with 32-bit offsets inside one row.  The CSR is read once per level and
// is about as large as the L2, so its loads are marked streaming (evicted
// first) and the W-word state arrays, gathered at random, keep the L2
// (headline kernel 0.844 -> 0.829 ms).
template <int U, bool kShared = false>
__device__ __forceinline__ void load_row(const int32_t *__restrict__ row, int x, int len,
                                         int stride, int (&c)[U])
{
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int ee = x + u * stride;
        c[u] = ee < len ? (kShared ? row[ee] : __ldcs(row + ee)) : -1;
    }
}

// Stage the column indices col[b, e) (e - b <= kChunk) into a warp's slot
// of kHubSlots entries in shared memory; returns the address of col[b]'s
// copy.  Called by the whole warp.  Whole 16-byte pieces inside the array
// go by cp.async; the at most 3 entries past the array's last whole piece
// by plain loads.
__device__ __forceinline__ const int32_t *stage_cols(int32_t *slot, const int32_t *col,
                                                     int64_t arcs, int64_t b, int64_t e,
                                                     int lane)
{
    const int64_t b4 = b & ~3ll;
    const int64_t e4 = min((e + 3) & ~3ll, arcs & ~3ll);
    for (int64_t x = b4 + 4 * lane; x < e4; x += 128) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(slot + (x - b4));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(col + x)
                     : "memory");
    }
    for (int64_t x = max(e4, b) + lane; x < e; x += 32) slot[x - b4] = col[x];
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
    return slot + (b - b4);
}

// OR of the frontier words (word w) of the neighbours col[base + off],
// col[base + off + stride], ... below e, U per step, until `done(acc)`
// holds, tested after every chk-th step (a later test only scans more).
// The step count depends on base, e, stride and `done` only, so it is
// uniform over lanes that share them (`done` may be warp-collective).  The
// column indices of the next step are loaded while the current frontier
// words are in flight: a step costs one dependent round trip, not two.
template <int W, int U, bool kShared = false, class Done>
__device__ __forceinline__ uint64_t gather_scan(const int32_t *__restrict__ col,
                                                const uint64_t *Fin, int64_t base, int off,
                                                int64_t e, int stride, int w,
                                                unsigned &words, int chk, Done done)
{
    // Offsets inside the row are 32-bit (a degree is below 2^31).
    const int32_t *row = col + base;
    const int len = (int)(e - base);
    uint64_t acc = 0;
    unsigned wl = 0;
    int c[U];
    load_row<U, kShared>(row, off, len, stride, c);
    int step = 0;
    for (int t = 0; t < len; t += U * stride) {
        int cn[U];
        load_row<U, kShared>(row, t + off + U * stride, len, stride, cn);
        acc |= gather_cols<W, U>(Fin, c, w, wl);
        if (++step == chk) {
            step = 0;
            if (done(acc)) break;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) c[u] = cn[u];
    }
    words += wl;
    return acc;
}

// Flush per-lane counters of one level phase to the level control block and
// (when asked) the CTA histogram to the global histogram of level l.
__device__ void flush_level(const BfsJob &J, int l, LevelCtl *C, LaneAcc &A,
                            unsigned *s_hist, bool flush_hist)
{
    __shared__ unsigned long long s_red[4][kBlock / 32];
    unsigned long long x[4] = {A.ef, A.eu_dec, A.ninc_dec, A.nfront};
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) x[q] += __shfl_xor_sync(FULL, x[q], o);
        if (lane == 0) s_red[q][wid] = x[q];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        unsigned long long t = 0;
        for (int i = 0; i < kBlock / 32; ++i) t += s_red[threadIdx.x][i];
        if (t) {
            if (threadIdx.x == 0) atomicAdd(&C->ef, t);
            if (threadIdx.x == 1) atomicAdd(&C->eu_dec, t);
            if (threadIdx.x == 2) atomicAdd(&C->ninc_dec, (unsigned)t);
            if (threadIdx.x == 3) atomicAdd(&C->qlen, (unsigned)t);
        }
    }
    A.ef = A.eu_dec = 0;
    A.ninc_dec = A.nfront = 0;
    if (!flush_hist) return;
    __syncthreads();
    for (int i = threadIdx.x; i < J.k; i += blockDim.x) {
        const unsigned c = s_hist[i];
        if (c) {
            atomicAdd(&J.hist[(int64_t)l * J.k + i], c);
            s_hist[i] = 0;
        }
    }
}

// Order-preserving stream compaction over [0, N) by all CTAs: each CTA
// takes a contiguous slice, counts its keepers, reserves their slots with
// one atomicAdd on *counter, then calls put(slot, i) for them in slice order.
template <class Keep, class Put>
__device__ void block_compact_put(int64_t N, Keep keep, Put put, unsigned *counter,
                                  unsigned team_rank, unsigned team_size)
{
    __shared__ unsigned s_w[kBlock / 32];
    __shared__ unsigned s_base;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t per = (N + team_size - 1) / team_size;
    const int64_t lo = (int64_t)team_rank * per, hi = min(N, lo + per);
    // keep(i) of this thread's first 32 entries, reused by the second sweep
    // (each test costs dependent loads).
    unsigned c = 0, kbits = 0;
    {
        int j = 0;
#pragma unroll 4
        for (int64_t i = lo + tid; i < hi; i += kBlock, ++j) {
            const bool k = keep(i);
            c += k ? 1u : 0u;
            if (k && j < 32) kbits |= 1u << j;
        }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if (lane == 0) s_w[wid] = c;
    __syncthreads();
    if (tid == 0) {
        unsigned t = 0;
        for (int i = 0; i < kBlock / 32; ++i) t += s_w[i];
        s_base = t ? atomicAdd(counter, t) : 0u;
    }
    __syncthreads();
    unsigned base = s_base;
    int j = 0;
    for (int64_t c0 = lo; c0 < hi; c0 += kBlock, ++j) {
        const int64_t i = c0 + tid;
        const bool k = i < hi && (j < 32 ? ((kbits >> j) & 1u) != 0u : keep(i));
        const unsigned bal = __ballot_sync(FULL, k);
        if (lane == 0) s_w[wid] = __popc(bal);
        __syncthreads();
        unsigned off = 0, tot = 0;
        for (int q = 0; q < kBlock / 32; ++q) {
            if (q < wid) off += s_w[q];
            tot += s_w[q];
        }
        if (k) put(base + off + __popc(bal & ((1u << lane) - 1u)), i);
        base += tot;
        __syncthreads();
    }
}

// The same, writing out[slot] = get(i).
template <class Keep, class Get>
__device__ void block_compact(int64_t N, Keep keep, Get get, int32_t *out, unsigned *counter,
                              unsigned team_rank, unsigned team_size)
{
    block_compact_put(
        N, keep, [&](unsigned slot, int64_t i) { out[slot] = get(i); }, counter, team_rank,
        team_size);
}

// Top-down push of one frontier node's words f (slot w per lane) to the
// CSR entries [b, e): new bits are OR-ed into nxt and each node reached for
// the first time this level is appended (once) to the touched list.  Called
// by a whole warp.  When every word has bits, lane groups of W take NPW
// entries per step; otherwise the words with bits are pushed one after
// another by all 32 lanes (a word per lane group would leave the lanes of
// empty words idle).  kUnroll entries per lane and step.
template <int W>
__device__ __forceinline__ void td_push(const BfsJob &J, const int32_t *__restrict__ col,
                                        uint64_t f, int64_t b, int64_t e, LevelCtl *C,
                                        int32_t *Tout, LaneAcc &A, const Stage &stage)
{
    constexpr int NPW = 32 / W;
    const int lane = threadIdx.x & 31;
    const int w = lane & (W - 1);
    const int grp = lane / W;
    const int32_t *row = col + b;
    const int len = (int)(e - b);
    unsigned wl = 0;
    const unsigned S = __ballot_sync(FULL, f != 0ull) &
                       (W == 32 ? 0xFFFFFFFFu : ((1u << W) - 1u));
    if (S == 0u) return;
    if (__popc(S) < W) {
        for (unsigned s = S; s; s &= s - 1) {
            const int ww = __ffs(s) - 1;
            const uint64_t fw = __shfl_sync(FULL, f, ww);
            int vn[kUnroll];
            load_row<kUnroll>(row, lane, len, 32, vn);
            for (int t = lane; t < len; t += 32 * kUnroll) {
                int vv[kUnroll];
                uint64_t vs[kUnroll];
#pragma unroll
                for (int q = 0; q < kUnroll; ++q) vv[q] = vn[q];
                load_row<kUnroll>(row, t + 32 * kUnroll, len, 32, vn);
#pragma unroll
                for (int q = 0; q < kUnroll; ++q)
                    vs[q] = vv[q] >= 0 ? J.vis[(int64_t)vv[q] * W + ww] : ~0ull;
#pragma unroll
                for (int q = 0; q < kUnroll; ++q) {
                    if (vv[q] < 0) continue;
                    const int v = vv[q];
                    wl += 1;
                    const uint64_t nbits = fw & ~vs[q];
                    if (!nbits) continue;
                    const uint64_t old =
                        atomicOr((unsigned long long *)&J.nxt[(int64_t)v * W + ww], nbits);
                    if (old == 0ull && atomicCAS(&J.tflag[v], 0u, 1u) == 0u)
                        stage_push(stage, v, Tout, &C->tlen);
                }
            }
        }
        A.words += wl;
        return;
    }
    // The next step's column indices load while this step's visited words
    // are in flight; offsets inside the row are 32-bit.
    int vn[kUnroll];
    load_row<kUnroll>(row, grp, len, NPW, vn);
    for (int t = grp; t < len; t += NPW * kUnroll) {
        int vv[kUnroll];
        uint64_t vs[kUnroll];
#pragma unroll
        for (int q = 0; q < kUnroll; ++q) vv[q] = vn[q];
        load_row<kUnroll>(row, t + NPW * kUnroll, len, NPW, vn);
#pragma unroll
        for (int q = 0; q < kUnroll; ++q)
            vs[q] = vv[q] >= 0 ? J.vis[(int64_t)vv[q] * W + w] : ~0ull;
#pragma unroll
        for (int q = 0; q < kUnroll; ++q) {
            if (vv[q] < 0) continue;
            const int v = vv[q];
            wl += 1;
            const uint64_t nbits = f & ~vs[q];
            if (!nbits) continue;
            const uint64_t old =
                atomicOr((unsigned long long *)&J.nxt[(int64_t)v * W + w], nbits);
            if (old == 0ull && atomicCAS(&J.tflag[v], 0u, 1u) == 0u)
                stage_push(stage, v, Tout, &C->tlen);
        }
    }
    A.words += wl;
}

// Top-down push of one low-degree frontier node by its lane group: lane w
// pushes word f (its word w) to the `len` entries of `row`, kUnroll entries
// per step (the column indices are the same for the group's lanes and load
// as one broadcast).  Same effect as td_push.
template <int W>
__device__ __forceinline__ void td_push_lane(const BfsJob &J, const int32_t *__restrict__ row,
                                             int len, uint64_t f, int w, LevelCtl *C,
                                             int32_t *Tout, LaneAcc &A, const Stage &stage)
{
    unsigned wl = 0;
    for (int x = 0; x < len; x += kUnroll) {
        int vv[kUnroll];
        load_row<kUnroll>(row, x, len, 1, vv);
        uint64_t vs[kUnroll];
#pragma unroll
        for (int q = 0; q < kUnroll; ++q)
            vs[q] = vv[q] >= 0 ? J.vis[(int64_t)vv[q] * W + w] : ~0ull;
#pragma unroll
        for (int q = 0; q < kUnroll; ++q) {
            if (vv[q] < 0) continue;
            const int v = vv[q];
            wl += 1;
            const uint64_t nbits = f & ~vs[q];
            if (!nbits) continue;
            const uint64_t old =
                atomicOr((unsigned long long *)&J.nxt[(int64_t)v * W + w], nbits);
            if (old == 0ull && atomicCAS(&J.tflag[v], 0u, 1u) == 0u)
                stage_push(stage, v, Tout, &C->tlen);
        }
    }
    A.words += wl;
}

// Active lists of the bottom-up levels (see bfs_pass).
struct ActiveLists {
    const int32_t *L, *M, *H, *HC, *T;
    const int4 *TA;
    int64_t nL, nM, nH, nHC, nT;
    int nextL, nextM, nextH, nextT;
};

// One traversal pass of job J on the team (team_rank, team_size); barriers
// on *bar.  On error (a barrier timed out) the pass returns early with the
// code in bar->err.
template <int W>
__device__ void bfs_pass(const BfsJob &J, unsigned team_rank, unsigned team_size, Ctl *bar,
                         unsigned *s_hist)
{
    constexpr int NPW = 32 / W;           // nodes (or entries) per warp step
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t gthreads = (int64_t)team_size * kBlock;
    const int64_t gtid = (int64_t)team_rank * kBlock + tid;
    const int64_t gwarp = gtid >> 5, nwarps = gthreads >> 5;
    const int w = lane & (W - 1);
    const int grp = lane / W;
    const int64_t n = J.n;
    const int64_t *rp = J.rp;
    const int32_t *col = J.col;
    const int64_t *prp = J.prp;
    const int32_t *pcol = J.pcol;
    Ctl *ctl = J.ctl;
    const unsigned nb = team_size;
    const bool doHist = (J.red & RED_HIST) != 0;

    // Top-down: the touched-list stage; bottom-up heavy tasks: each warp's
    // staged column indices (kHubSlots entries) for W <= 8 (wider variants
    // keep their shared memory for the histogram, within the 25 % carveout
    // a server gives every traversal variant at 4 CTAs/SM).
    constexpr bool kStageHub = CC_MSBFS_STAGE && W <= 8;
    constexpr int kHubN = kStageHub ? (kBlock / 32) * kHubSlots : 0;
    constexpr int kBufN = kStage > kHubN ? kStage : kHubN;
    __shared__ __align__(16) int32_t s_buf[kBufN];
    __shared__ unsigned s_cnt, s_base;
    const Stage stage{s_buf, &s_cnt, &s_base};
    if (threadIdx.x == 0) s_cnt = 0;

    // Warp time per phase (tracing): lane 0 of each warp adds the clock
    // cycles since its previous lap to the CTA's counter of the phase that
    // just ended; waits in the grid barrier count as CC_PH_BARRIER.
    __shared__ unsigned long long s_ph[CC_NUM_PHASES];
    if (threadIdx.x < CC_NUM_PHASES) s_ph[threadIdx.x] = 0;
    __syncthreads();
    long long ph_t = clock64();
    auto lap = [&](int p) {
        const long long t = clock64();
        if (lane == 0) atomicAdd(&s_ph[p], (unsigned long long)(t - ph_t));
        ph_t = t;
    };
    auto sync_after = [&](int p) {
        lap(p);
        const bool ok = grid_sync(bar, team_rank, nb, J.timeout_ns);
        lap(CC_PH_BARRIER);
        return ok;
    };

    LaneAcc A;
    A.ef = A.eu_dec = A.words = 0;
    A.ninc_dec = A.nfront = 0;

    if (J.gate && J.gate[0] == 0u && J.gate[1] == 0u) return;  // uniform: no barrier yet

    // ---- level 0: clear the state, seed the sources -----------------------
    for (int64_t i = gtid; i < n * W; i += gthreads) {
        J.vis[i] = pad_mask(J.k, (int)(i & (W - 1)));
        J.F0[i] = 0;
        J.F1[i] = 0;
        J.nxt[i] = 0;
    }
    for (int64_t v = gtid; v < n; v += gthreads) {
        J.tflag[v] = 0;
        J.fstamp[v] = kInf;
    }
    for (int i = tid; i < W * 64; i += kBlock) s_hist[i] = 0;
    if (J.red & RED_LC)
        for (int64_t i = gtid; i < 2 * n; i += gthreads) J.lc2[i] = 0;
    if (J.red & RED_BAND)
        for (int64_t v = gtid; v < n; v += gthreads) J.bflag[v] = 0;
    if (J.red & RED_LEVELS)
        for (int64_t i = gtid; i < n * J.dist_ld; i += gthreads) J.dist_out[i] = kInf;
    if (!sync_after(CC_PH_INIT)) return;
    for (int64_t i = gtid; i < J.k; i += gthreads) {
        const int v = J.sources[i];
        const uint64_t bit = 1ull << (i & 63);
        const int64_t vw = (int64_t)v * W + (i >> 6);
        atomicOr((unsigned long long *)&J.vis[vw], bit);
        atomicOr((unsigned long long *)&J.F0[vw], bit);
        J.fstamp[v] = 0u;
        if (J.red & RED_LEVELS) J.dist_out[(int64_t)v * J.dist_ld + i] = 0u;
        if (J.red & RED_PIVOT) { J.pivot[v] = (int)i; J.delta[v] = 0; }
        if (J.red & RED_DCC) J.dcc[i * J.dcc_k + J.sidx[v]] = 0;
        const unsigned long long d = (unsigned long long)(rp[v + 1] - rp[v]);
        atomicAdd(&ctl->lev[0].ef, d);
        if (J.k == 1) {
            atomicAdd(&ctl->lev[0].eu_dec, d);
            atomicAdd(&ctl->lev[0].ninc_dec, 1u);
        }
    }
    if (gtid == 0) {
        ctl->lev[0].qlen = (unsigned)J.k;
        ctl->lev[0].tlen = (unsigned)J.k;  // level 0 "touched" the sources
    }
    if (!sync_after(CC_PH_INIT)) return;

    long long eu = J.arcs, ninc = n;
    int last = 0;
    // Active lists of the bottom-up levels: the light, medium and heavy
    // node lists and the heavy chunk tasks (null: all), later rebuilt
    // (order-preserving) into AL0 / AL1 and ACH0 / ACH1 once the incomplete
    // nodes fall below half of them; the tiny nodes' list and inline
    // neighbours, compacted together.  The same for the whole CTA and live
    // through the pass, they sit in shared memory, out of the registers the
    // scans need; thread 0 updates them between block barriers.
    __shared__ ActiveLists s_al;
    if (tid == 0) {
        s_al.L = J.Llist; s_al.M = J.Mlist; s_al.H = J.Hlist; s_al.HC = nullptr;
        s_al.T = J.Tlist; s_al.TA = J.Tadj;
        s_al.nL = J.nL; s_al.nM = J.nM; s_al.nH = J.nH; s_al.nHC = J.nHch; s_al.nT = J.nT;
        s_al.nextL = s_al.nextM = s_al.nextH = s_al.nextT = 0;
    }
    __syncthreads();
    // Queue of a top-down level: the previous level's touched list when that
    // level was top-down (level 0 "touched" the sources), else built from
    // the frontier stamps.
    bool prev_td = true;
    const int32_t *prevT = J.sources;
    int l = 1;
    for (;; ++l) {
        volatile LevelCtl *P = &ctl->lev[(l - 1) & 3];
        const unsigned qprev = P->qlen;
        const unsigned tprev = P->tlen;
        const unsigned long long ef = P->ef;
        eu -= (long long)P->eu_dec;
        // The warp-wide completion test of the medium and heavy scans (a
        // shuffle reduction) runs every 4th step while the last level
        // completed no node, every step once nodes complete.
        const int chk = P->ninc_dec == 0 ? 4 : 1;
        ninc -= (long long)P->ninc_dec;
        if (qprev > 0) last = l - 1;
        if (qprev == 0 || ninc == 0) break;
        if (doHist && l >= J.hist_cap) {
            if (gtid == 0) atomicCAS(&ctl->err, 0, 1);  // histogram too short
            break;
        }
        const bool td = ef * (unsigned long long)J.alpha < (unsigned long long)eu;
        if (gtid == 0 && l < kTraceLevels) {
            ctl->lvl_ns[l] = gtimer();
            ctl->lvl_td[l] = td;
            ctl->lvl_front[l] = qprev;
            ctl->lvl_ef[l] = ef;
        }
        if (gtid == 0) {
            LevelCtl *Z = &ctl->lev[(l + 1) & 3];
            Z->qlen = 0; Z->tlen = 0; Z->ninc_dec = 0; Z->ef = 0; Z->eu_dec = 0;
            Z->alen = 0; Z->qcnt = 0; Z->mlen = 0; Z->hlen = 0; Z->hclen = 0; Z->tlen2 = 0;
            Z->hnext = 0;
        }
        uint64_t *Fin = (l & 1) ? J.F0 : J.F1;
        uint64_t *Fout = (l & 1) ? J.F1 : J.F0;
        LevelCtl *C = &ctl->lev[l & 3];

        if (td) {
            const int32_t *Qin = prevT;
            int64_t qn = tprev;
            if (!prev_td) {
                const unsigned want = (unsigned)(l - 1);
                block_compact(
                    n, [&](int64_t i) { return J.fstamp[i] == want; },
                    [&](int64_t i) { return (int32_t)i; }, J.Q0, &C->qcnt, team_rank, team_size);
                if (!sync_after(CC_PH_TD_QUEUE)) return;
                Qin = J.Q0;
                qn = ((volatile LevelCtl *)C)->qcnt;
            }
            int32_t *Tout = (Qin == J.T) ? J.Q1 : J.T;
            // P1: push the frontier words of the queued nodes.  A frontier
            // of at most one node per warp: each node's entries split over
            // S = nwarps / qn warps, so that the level takes one push step
            // where a warp per node took several (heavy nodes pushed by
            // their chunk tasks below).
            const bool few = qn <= nwarps;
            const int64_t S = few && qn > 0 ? nwarps / qn : 1;
            for (int64_t t = gwarp; few && t < qn * S; t += nwarps) {
                const int u = Qin[t / S];
                const int64_t part = t % S;
                const int64_t b = rp[u], e = rp[u + 1];
                if (J.ntH > 0 && e - b > kMediumMaxDeg) continue;
                const int64_t per = (e - b + S - 1) / S;
                const int64_t bb = b + part * per, ee = min(e, bb + per);
                if (bb >= ee) continue;
                const uint64_t f = Fin[(int64_t)u * W + w];
                td_push<W>(J, col, f, bb, ee, C, Tout, A, stage);
            }
            // Otherwise nodes of at most kLightMaxDeg entries: a lane group
            // each, NPW per warp (a grid's frontier node has 4 entries: a
            // warp each would leave most lanes idle and chain one node after
            // another).
            for (int64_t t0 = gwarp * NPW; !few && t0 < qn; t0 += nwarps * NPW) {
                const int64_t t = t0 + grp;
                if (t < qn) {
                    const int u = Qin[t];
                    const int64_t b = rp[u], e = rp[u + 1];
                    if (e - b <= kLightMaxDeg) {
                        const uint64_t f = Fin[(int64_t)u * W + w];
                        if (f) td_push_lane<W>(J, col + b, (int)(e - b), f, w, C, Tout, A, stage);
                    }
                }
            }
            // Larger nodes: a warp tests its queue entries (every nwarps-th,
            // so that consecutive ones go to different warps) 32 at a time
            // by ballot and pushes each larger one whole; when the graph has
            // chunk tasks, a heavy node's list is pushed by them.
            for (int64_t j0 = 0; !few && gwarp + j0 * nwarps < qn; j0 += 32) {
                const int64_t t = gwarp + (j0 + lane) * nwarps;
                int u = 0;
                int64_t b = 0, e = 0;
                bool big = false;
                if (t < qn) {
                    u = Qin[t];
                    b = rp[u];
                    e = rp[u + 1];
                    big = e - b > kLightMaxDeg && !(J.ntH > 0 && e - b > kMediumMaxDeg);
                }
                unsigned m = __ballot_sync(FULL, big);
                while (m) {
                    const int src = __ffs(m) - 1;
                    m &= m - 1;
                    const int uu = __shfl_sync(FULL, u, src);
                    const int64_t bb = __shfl_sync(FULL, b, src);
                    const int64_t ee = __shfl_sync(FULL, e, src);
                    const uint64_t f = Fin[(int64_t)uu * W + w];
                    td_push<W>(J, col, f, bb, ee, C, Tout, A, stage);
                }
            }
            // Heavy frontier nodes: the warp's chunk tasks (every nwarps-th)
            // are tested 32 at a time, a lane each, and only those of nodes
            // that gained bits last level are pushed, by the whole warp.
            for (int64_t j0 = 0; gwarp + j0 * nwarps < J.ntH; j0 += 32) {
                const int64_t t = gwarp + (j0 + lane) * nwarps;
                int u = 0;
                bool act = false;
                if (t < J.ntH) {
                    u = J.tHn[t];
                    act = J.fstamp[u] == (unsigned)(l - 1);
                }
                unsigned m = __ballot_sync(FULL, act);
                while (m) {
                    const int src = __ffs(m) - 1;
                    m &= m - 1;
                    const int uu = __shfl_sync(FULL, u, src);
                    const uint64_t f = Fin[(int64_t)uu * W + w];
                    if (__all_sync(FULL, f == 0ull)) continue;
                    const int64_t b = J.tHb[gwarp + (j0 + src) * nwarps];
                    td_push<W>(J, col, f, b, min(b + (int64_t)kChunk, rp[uu + 1]), C, Tout,
                               A, stage);
                }
            }
            stage_flush(stage, Tout, &C->tlen);
            if (!sync_after(CC_PH_TD_PUSH)) return;
            // P2: finalise the touched nodes.
            const int64_t tl = ((volatile LevelCtl *)C)->tlen;
            for (int64_t t = gwarp; t * NPW < tl; t += nwarps) {
                const int64_t li = t * NPW + grp;
                const bool valid = li < tl;
                const int v = valid ? Tout[li] : 0;
                const int64_t vw = (int64_t)v * W + w;
                uint64_t vis = ~0ull, acc = 0;
                int64_t deg = 0;
                if (valid) {
                    vis = J.vis[vw];
                    acc = J.nxt[vw];
                    if (acc) J.nxt[vw] = 0;
                    deg = prp[v + 1] - prp[v];
                }
                tile_reduce<W>(J, l, valid, v, vis, acc & ~vis, deg, Fout, A, s_hist, true);
            }
            flush_words(ctl, l, A.words);
            A.words = 0;
            flush_level(J, l, C, A, s_hist, doHist);
            if (!sync_after(CC_PH_TD_FINAL)) return;
            if (gtid == 0) ctl->td_levels += 1;
            prev_td = true;
            prevT = Tout;
        } else {
            // Rebuild the light list when fewer than half of it can still be
            // incomplete (ninc bounds the incomplete light nodes).
            // ninc bounds the incomplete nodes of every class; the medium and
            // heavy lists are rebuilt with the light list (heavy nodes complete
            // early) or on their own bound.
            // The tiny and light lists are rebuilt together, once fewer than
            // half of their entries can still be incomplete.
            const bool rb_tl = 2 * ninc < s_al.nL + s_al.nT;
            const bool rb_t = rb_tl && s_al.nT > 0;
            const bool rb_l = rb_tl && s_al.nL > 0;
            const bool rb_m = s_al.nM > 0 && (rb_l || 2 * ninc < s_al.nM);
            const bool rb_h = s_al.nH > 0 && (rb_l || 2 * ninc < s_al.nH);
            if (rb_t || rb_l || rb_m || rb_h) {
                auto incomplete = [&](int64_t v) {
                    bool inc = false;
                    for (int q = 0; q < W; ++q) inc |= J.vis[v * W + q] != ~0ull;
                    return inc;
                };
                // Lists are compacted into the buffer of the other parity
                // (next*); the new heads and lengths are set after the barrier.
                int32_t *const tout = s_al.nextT ? J.AT1 : J.AT0;
                int4 *const taout = s_al.nextT ? J.ATa1 : J.ATa0;
                int32_t *const lout = s_al.nextL ? J.AL1 : J.AL0;
                int32_t *const mout = (s_al.nextM ? J.AL1 : J.AL0) + J.nL;
                int32_t *const hout = (s_al.nextH ? J.AL1 : J.AL0) + J.nL + J.nM;
                int32_t *const cout = s_al.nextH ? J.ACH1 : J.ACH0;
                if (rb_t) {
                    const int32_t *in = s_al.T;
                    const int4 *ain = s_al.TA;
                    block_compact_put(
                        s_al.nT, [&](int64_t i) { return incomplete(in[i]); },
                        [&](unsigned slot, int64_t i) {
                            tout[slot] = in[i];
                            taout[slot] = ain[i];
                        },
                        &C->tlen2, team_rank, team_size);
                }
                if (rb_l) {
                    const int32_t *in = s_al.L;
                    block_compact(
                        s_al.nL, [&](int64_t i) { return incomplete(in[i]); },
                        [&](int64_t i) { return in[i]; }, lout, &C->alen, team_rank, team_size);
                }
                if (rb_m) {
                    const int32_t *in = s_al.M;
                    block_compact(
                        s_al.nM, [&](int64_t i) { return incomplete(in[i]); },
                        [&](int64_t i) { return in[i]; }, mout, &C->mlen, team_rank, team_size);
                }
                if (rb_h) {
                    const int32_t *in = s_al.H;
                    block_compact(
                        s_al.nH, [&](int64_t i) { return incomplete(in[i]); },
                        [&](int64_t i) { return in[i]; }, hout, &C->hlen, team_rank, team_size);
                    const int32_t *cin = s_al.HC;
                    block_compact(
                        s_al.nHC,
                        [&](int64_t i) {
                            return incomplete(J.Hch_node[cin ? cin[i] : (int32_t)i]);
                        },
                        [&](int64_t i) { return cin ? cin[i] : (int32_t)i; }, cout, &C->hclen,
                        team_rank, team_size);
                }
                if (!sync_after(CC_PH_BU_REBUILD)) return;
                if (tid == 0) {
                    const volatile LevelCtl *VC = C;
                    if (rb_t) {
                        s_al.T = tout; s_al.TA = taout; s_al.nT = VC->tlen2; s_al.nextT ^= 1;
                    }
                    if (rb_l) { s_al.L = lout; s_al.nL = VC->alen; s_al.nextL ^= 1; }
                    if (rb_m) { s_al.M = mout; s_al.nM = VC->mlen; s_al.nextM ^= 1; }
                    if (rb_h) {
                        s_al.H = hout; s_al.nH = VC->hlen;
                        s_al.HC = cout; s_al.nHC = VC->hclen; s_al.nextH ^= 1;
                    }
                }
                __syncthreads();
            }
            // A0: tiny nodes, one thread per (node, word); the neighbours come
            // with the list entry, so every frontier word is gathered at once.
            // The next tile's entries load while this tile's words are in
            // flight.
            const int32_t *const TLcur = s_al.T;
            const int4 *const TAcur = s_al.TA;
            const int64_t tl_len = s_al.nT;
            int vnext = 0;
            int4 nbnext = make_int4(-1, -1, -1, -1);
            if (gwarp * NPW + grp < tl_len) {
                vnext = TLcur[gwarp * NPW + grp];
                nbnext = TAcur[gwarp * NPW + grp];
            }
            for (int64_t t = gwarp; t * NPW < tl_len; t += nwarps) {
                const int64_t li = t * NPW + grp;
                const bool valid = li < tl_len;
                const int v = vnext;
                const int4 nb = nbnext;
                const int64_t ln = li + nwarps * NPW;
                if (ln < tl_len) {
                    vnext = TLcur[ln];
                    nbnext = TAcur[ln];
                }
                const int64_t vw = (int64_t)v * W + w;
                const uint64_t vis = valid ? J.vis[vw] : ~0ull;
                const int deg = (nb.x >= 0) + (nb.y >= 0) + (nb.z >= 0) + (nb.w >= 0);
                uint64_t acc = 0;
                if (vis != ~0ull) {
                    const int c4[4] = {nb.x, nb.y, nb.z, nb.w};
                    unsigned wl = 0;
                    acc = gather_cols<W, 4>(Fin, c4, w, wl);
                    A.words += wl;
                }
                __syncwarp();
                tile_reduce<W>(J, l, valid, v, vis, acc & ~vis, deg, Fout, A, s_hist, false);
            }
            // A1: light nodes of the active list, one thread per (node, word).
            const int32_t *const ALcur = s_al.L;
            const int64_t al_len = s_al.nL;
            int anext = gwarp * NPW + grp < al_len ? ALcur[gwarp * NPW + grp] : 0;
            for (int64_t t = gwarp; t * NPW < al_len; t += nwarps) {
                const int64_t li = t * NPW + grp;
                const bool valid = li < al_len;
                const int v = valid ? anext : 0;
                if (li + nwarps * NPW < al_len) anext = ALcur[li + nwarps * NPW];
                const int64_t vw = (int64_t)v * W + w;
                uint64_t vis = valid ? J.vis[vw] : ~0ull;
                int64_t b = 0, e = 0;
                if (valid) { b = prp[v]; e = prp[v + 1]; }
                uint64_t acc = 0;
                if (vis != ~0ull)
                    acc = gather_scan<W, kUnroll>(pcol, Fin, b, 0, e, 1, w, A.words, 1,
                                                  [&](uint64_t a) { return (a | vis) == ~0ull; });
                __syncwarp();
                tile_reduce<W>(J, l, valid, v, vis, acc & ~vis, e - b, Fout, A, s_hist,
                               false);
            }
            lap(CC_PH_BU_LIGHT);
            // A2: medium nodes, a warp per node.  The warp scans NPW of its
            // nodes one after another, lane group g keeping node g's words,
            // then one fused reduction covers all NPW.
            const int32_t *const MLcur = s_al.M;
            const int64_t ml_len = s_al.nM;
            for (int64_t t0 = gwarp; t0 < ml_len; t0 += (int64_t)NPW * nwarps) {
                int myv = 0;
                uint64_t myvis = ~0ull, myres = 0;
                int64_t mydeg = 0;
                bool myvalid = false;
                for (int g = 0; g < NPW; ++g) {
                    const int64_t t = t0 + (int64_t)g * nwarps;
                    if (t >= ml_len) break;
                    const int v = MLcur[t];
                    const uint64_t visw = J.vis[(int64_t)v * W + w];
                    const int64_t b = prp[v], e = prp[v + 1];
                    uint64_t r = 0;
                    if (!__all_sync(FULL, visw == ~0ull)) {
                        const uint64_t acc = gather_scan<W, kUnrollM>(
                            pcol, Fin, b, grp, e, NPW, w, A.words, chk, [&](uint64_t a) {
                                return __all_sync(FULL, (or_same_word<W>(a) | visw) == ~0ull);
                            });
                        r = or_same_word<W>(acc);
                    }
                    if (grp == g) {
                        myv = v;
                        myvis = visw;
                        myres = r;
                        mydeg = e - b;
                        myvalid = true;
                    }
                }
                tile_reduce<W>(J, l, myvalid, myv, myvis, myres & ~myvis, mydeg, Fout, A,
                               s_hist, false);
            }
            lap(CC_PH_BU_MEDIUM);
            // A3: heavy nodes, 256-entry warp tasks OR-ing into nxt.  Read in
            // place, a task's column indices would stream from DRAM one
            // 128-byte line per scan step (the CSR does not stay in the L2):
            // a task that still scans stages its chunk of the hub's adjacency
            // in the warp's slice of shared memory first (W <= 8) or
            // prefetches its lines to the L2 (wider variants), so that a
            // step waits only for its frontier gathers (headline traversal:
            // prefetch 0.831 -> 0.803 ms, staging instead 0.779 -> 0.763).
            const int32_t *const HCcur = s_al.HC;
            const int64_t hc_len = s_al.nHC;
            auto heavy_task = [&](int64_t t) {
                const int32_t ti = HCcur ? HCcur[t] : (int32_t)t;
                const int v = J.Hch_node[ti];
                const int64_t vw = (int64_t)v * W + w;
                const int64_t b = J.Hch_begin[ti];
                const int64_t e = min(b + (int64_t)kChunk, prp[v + 1]);
                const uint64_t visw = J.vis[vw];
                const uint64_t cur = J.nxt[vw];
                if (__all_sync(FULL, (visw | cur) == ~0ull)) return;
                auto done = [&](uint64_t a) {
                    return __all_sync(FULL, (or_same_word<W>(a) | visw | cur) == ~0ull);
                };
                uint64_t acc;
                if constexpr (kStageHub) {
                    const int32_t *srow = stage_cols(s_buf + (threadIdx.x >> 5) * kHubSlots,
                                                     pcol, J.arcs, b, e, lane);
                    acc = gather_scan<W, kUnrollH, true>(srow, Fin, 0, grp, e - b, NPW, w,
                                                         A.words, chk, done);
                } else {
                    if (lane <= kChunk / 32) prefetch_l2(pcol + min(b + 32 * lane, e - 1));
                    acc = gather_scan<W, kUnrollH>(pcol, Fin, b, grp, e, NPW, w, A.words, chk,
                                                   done);
                }
                const uint64_t nbits = or_same_word<W>(acc) & ~visw & ~cur;
                if (lane < W && nbits) atomicOr((unsigned long long *)&J.nxt[vw], nbits);
            };
            if (hc_len > 2 * nwarps) {
                // Many tasks: the warps take them from a counter, kGrab at a
                // time, so that warps done early with the other classes take
                // more of them (dealt in turn, the level waits for the warp
                // with the most work; 0.803 -> 0.789 ms).
                for (;;) {
                    unsigned tb = 0;
                    if (lane == 0) tb = atomicAdd(&C->hnext, (unsigned)kGrab);
                    tb = __shfl_sync(FULL, tb, 0);
                    if ((int64_t)tb >= hc_len) break;
                    const int64_t tend = min((int64_t)tb + kGrab, hc_len);
                    for (int64_t t = tb; t < tend; ++t) heavy_task(t);
                }
            } else {
                for (int64_t t = gwarp; t < hc_len; t += nwarps) heavy_task(t);
            }
            if (!sync_after(CC_PH_BU_HEAVY)) return;
            // B: finalise the heavy nodes.
            const int32_t *const HLcur = s_al.H;
            const int64_t hl_len = s_al.nH;
            for (int64_t t = gwarp; t * NPW < hl_len; t += nwarps) {
                const int64_t li = t * NPW + grp;
                const bool valid = li < hl_len;
                const int v = valid ? HLcur[li] : 0;
                const int64_t vw = (int64_t)v * W + w;
                uint64_t vis = ~0ull, acc = 0;
                int64_t deg = 0;
                if (valid) {
                    vis = J.vis[vw];
                    acc = J.nxt[vw];
                    if (acc) J.nxt[vw] = 0;
                    deg = prp[v + 1] - prp[v];
                }
                tile_reduce<W>(J, l, valid, v, vis, acc & ~vis, deg, Fout, A, s_hist, false);
            }
            flush_words(ctl, l, A.words);
            A.words = 0;
            flush_level(J, l, C, A, s_hist, doHist);
            if (!sync_after(CC_PH_BU_FINAL)) return;
            if (gtid == 0) ctl->bu_levels += 1;
            prev_td = false;
        }
    }
    // Pass statistics.
    if (tid < CC_NUM_PHASES) atomicAdd(&ctl->ph_cycles[tid], s_ph[tid]);
    if (gtid == 0) {
        ctl->levels = last;
        ctl->ninc_final = ninc;
        ctl->lvl_ns[l < kTraceLevels ? l : kTraceLevels] = gtimer();
    }
}

}  // namespace
}  // namespace ccg
