// Internal declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/cc.h"

namespace ccg {

constexpr int kBlock = 256;          // threads per CTA of the traversal kernel
// Degree classes of the traversal (build-time tunables).
// Medium nodes (a warp each, no chunk tasks) up to 256 arcs: headline
// traversal 0.761 ms at 128, 0.740-0.747 at 256 and 384, 0.755 at 512.
#ifndef CC_MEDIUM_MAX_DEG
#define CC_MEDIUM_MAX_DEG 256
#endif
#ifndef CC_CHUNK
#define CC_CHUNK 256
#endif
#ifndef CC_TINY_MAX_DEG
#define CC_TINY_MAX_DEG 4
#endif
constexpr int kTinyMaxDeg = CC_TINY_MAX_DEG;     // neighbours inline (one int4)
constexpr int kLightMaxDeg = 32;                 // thread-per-(node, word) scan
constexpr int kMediumMaxDeg = CC_MEDIUM_MAX_DEG;  // warp-per-node scan
constexpr int kChunk = CC_CHUNK;                 // CSR entries per heavy-node warp task
constexpr uint32_t kInf = 0xFFFFFFFFu;

// Reductions a traversal pass performs (bit set).
enum : uint32_t {
    RED_SUM = 1u,    // sum[v] += d, sumsq[v] += d^2
    RED_PIVOT = 2u,  // first arrival: pivot[v], delta[v]
    RED_DCC = 4u,    // delta_cc[i][j] for sampled nodes
    RED_HIST = 8u,   // per-source level histogram over V \ C
    RED_LC = 16u,    // hybrid pass: lc[v] += d, d^2 over sources in Lmask(v)
    RED_LEVELS = 32u, // dist_out[v * dist_ld + i] = level of v from source i
    // hybrid pass with the error estimate: for nodes flagged in sqflag,
    // hcse[v] += (d(c_i, v) - d(c(v), c_i))^2 over c_i beyond the threshold
    // (flag 1: not in Lmask; 128-bit {lo, hi}), and fdist[v] = d(c_i, v) for
    // c_i = istar[c(v)] (flag 2: no sampled node beyond the threshold)
    RED_SQ = 64u,
    // hybrid within the first pass (eps = eps_a / eps_b): a bit arriving at
    // node v on level l belongs to L(v) when (l + Delta(v)) eps_a <=
    // Delta(v) eps_b, to HC(v) when (l - Delta(v)) eps_a > Delta(v) eps_b --
    // lc2[v] += l, l^2 (the complement of L, turned into L's sums after the
    // pass; valid once bflag[v] & 2) --, and is deferred otherwise: its
    // level's offset in that band, l + Delta(v) - floor(Delta(v) eps_b /
    // eps_a), goes to band[v * 64W + i] (valid once bflag[v] & 1)
    RED_BAND = 128u,
};

// Per-level statistics, indexed by level mod 4 (written during level l,
// read during l+1 and l+2, cleared during l+3).
struct LevelCtl {
    unsigned int qlen;          // nodes with new bits this level (queue length)
    unsigned int tlen;          // touched nodes (top-down)
    unsigned int ninc_dec;      // nodes that became complete this level
    unsigned int alen;          // rebuilt light list length (bottom-up)
    unsigned int qcnt;          // frontier queue built from the stamps (top-down)
    unsigned int mlen;          // rebuilt medium list length (bottom-up)
    unsigned int hlen;          // rebuilt heavy list length (bottom-up)
    unsigned int hclen;         // rebuilt heavy chunk list length (bottom-up)
    unsigned int tlen2;         // rebuilt tiny list length (bottom-up)
    unsigned int hnext;         // next heavy chunk task to take (bottom-up)
    unsigned long long ef;      // sum of degrees of the frontier nodes
    unsigned long long eu_dec;  // sum of degrees of nodes completed
};

constexpr int kTraceLevels = 64;

struct Ctl {
    unsigned long long bar_arrive;  // grid barrier arrivals (see barrier.cuh)
    int err;                // 0 or a CC_ERR_* code
    int band_ovf;           // RED_BAND: some band offset did not fit a byte
    unsigned far_len[3];    // shortest paths: lengths of the three far queues
    unsigned long long far_min[3];  // and the smallest label each waits with
    int levels;             // last level that produced new bits
    long long ninc_final;   // nodes never completed (non-zero: disconnected)
    unsigned long long td_levels, bu_levels;
    unsigned long long edges, words;  // CSR entries examined, words gathered
    LevelCtl lev[4];
    // Trace of the first kTraceLevels levels: global timer at the start of
    // each level (and at the end of the pass), direction and frontier size.
    unsigned long long lvl_ns[kTraceLevels + 1];
    unsigned int lvl_td[kTraceLevels];
    unsigned int lvl_front[kTraceLevels];
    unsigned long long lvl_ef[kTraceLevels];
    unsigned long long lvl_words[kTraceLevels];
    // Warp clock cycles spent in each CC_PH_* phase over the pass.
    unsigned long long ph_cycles[CC_NUM_PHASES];
};

// One traversal pass over one graph.
struct BfsJob {
    int64_t n, arcs;
    // Top-down pushes along (rp, col) -- the arcs leaving a node -- with
    // 256-arc tasks (tHn, tHb) for its heavy nodes; bottom-up pulls along
    // (prp, pcol) -- the arcs entering a node -- whose degree classes are
    // Llist/Mlist/Hlist/Hch.  Both are the same CSR for undirected graphs.
    const int64_t *rp;
    const int32_t *col;
    const int32_t *tHn;
    const int64_t *tHb;
    int64_t ntH;
    const int64_t *prp;
    const int32_t *pcol;
    int k;                  // sources in this pass
    const int32_t *sources; // k node ids
    const int32_t *sidx;    // n: sample index or -1 (pass-level sample)
    const int32_t *Llist, *Mlist, *Hlist;
    int64_t nL, nM, nH;
    const int32_t *Hch_node;
    const int64_t *Hch_begin;
    int64_t nHch;
    uint64_t *vis, *F0, *F1, *nxt;  // n*W words each
    int32_t *Q0, *Q1, *T;           // n each
    // n each: active node lists of the bottom-up levels, light nodes from
    // entry 0, medium from nL, heavy from nL + nM.
    int32_t *AL0, *AL1;
    int32_t *ACH0, *ACH1;           // nHch each: active heavy chunk tasks
    // Tiny nodes (degree <= kTinyMaxDeg, pull side) with their neighbours
    // inline, and the active copies of both.
    const int32_t *Tlist;
    const int4 *Tadj;
    int64_t nT;
    int32_t *AT0, *AT1;             // nT each
    int4 *ATa0, *ATa1;              // nT each
    uint32_t *fstamp;               // n: last level a node got new bits
    unsigned int *tflag;            // n
    uint32_t red;
    uint64_t *sum2;      // n x 2: {sum, sumsq}
    int32_t *pivot;      // n
    uint32_t *delta;     // n
    uint32_t *dcc;       // dcc_k x dcc_k (row = source index)
    int dcc_k;
    uint32_t *hist;      // hist_cap x k (level-major)
    int hist_cap;
    const uint64_t *Lmask;  // n*W
    uint64_t *lc2;          // n x 2: {LCsum, LCsumSq}; zeroed by the pass (RED_LC)
    // When set, the pass does nothing if gate[0] = gate[1] = 0 (the hybrid
    // preparation found no node needing the second pass).
    const unsigned *gate;
    uint32_t *dist_out;     // RED_LEVELS: n x dist_ld chunk of levels
    int dist_ld;            // RED_LEVELS: row stride of dist_out (>= k)
    const uint8_t *sqflag;  // RED_SQ: per node, 1 = accumulate hcse, 2 = record fdist
    const int32_t *istar;   // RED_SQ: per sample index, the farthest other sample
    uint64_t *hcse;         // RED_SQ: n x 2
    uint32_t *fdist;        // RED_SQ: n
    uint8_t *band;          // RED_BAND: n x 64W band offsets of deferred bits
    uint8_t *bflag;         // RED_BAND: n, zeroed by the pass
    uint32_t eps_a, eps_b;  // RED_BAND: eps
    Ctl *ctl;
    uint64_t timeout_ns;
    int alpha;              // top-down while ef * alpha < eu
    int max_ctas;           // 0: a whole-GPU launch; else at most this many CTAs
};

// Launch one cooperative traversal pass (W = words per node, power of two
// in [1, 32]).  Returns a CC_* status of the launch itself.
int launch_msbfs(int W, const BfsJob &job, cudaStream_t st, int *grid_used);

int launch_barrier_selftest(uint64_t timeout_ns, int *err_out);

// A failed CUDA runtime call (before it is turned into CC_ERR_CUDA): named
// on stderr with its place when the environment sets CC_DEBUG.
void note_cuda_error(cudaError_t e, const char *file, int line);
int msbfs_min_blocks_per_sm();
int mssp_blocks_per_sm();
void msbfs_set_carveout(int percent);
void mssp_set_carveout(int percent);

// Device view of a resident graph (forward CSR and its degree classes).
struct GraphView {
    int64_t n, arcs;
    bool directed, weighted;
    const int64_t *rp;
    const int32_t *col;
    const int32_t *L, *M, *H, *Hn, *T;
    const int4 *Tadj;
    const int64_t *Hb;
    int64_t nL, nM, nH, nHch, nT;
    int alpha;
};
int graph_view(cc_graph_t g, GraphView *v);
// Default direction switch of the bit-packed traversal (alpha of
// cc_set_tuning) for W words per node.  Direction threshold: top-down while
// frontier arcs x alpha < arcs of incomplete nodes.  Measured (device time
// of one pass): a one-word sample prefers 6 on graphs of mean degree >= 8
// (R-MAT) and 14 on low-degree grids and meshes (512^2 grid, k = 64: 23 ms
// against 27 ms at 4); wider samples prefer 14 on R-MAT and 4 on low-degree
// graphs, whose frontier nodes push in lane groups (1024^2 grid, k = 256:
// 108 ms against 132 ms at 14; 886^2, k = 512: 160 ms against 183 ms).
inline int default_alpha(int W, int64_t n, int64_t arcs)
{
    const bool dense = arcs >= 8 * n;
    if (W == 1) return dense ? 6 : 14;
    return dense ? 14 : 4;
}

// Output number c of the splitmix64 stream `seed` (Steele, Lea and Flood
// 2014): the counter-based generator of the samplers.
__device__ __forceinline__ uint64_t splitmix64_out(uint64_t seed, uint64_t c)
{
    uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// Server slots: an empty handle whose workspace persists, pointed at the
// resident CSR of another handle per request.
cc_graph_t graph_new_empty();
int graph_borrow(cc_graph_t dst, cc_graph_t src);
size_t graph_workspace_bytes(cc_graph_t g);
// Estimates from the first pass resident in g's workspace (see cc_api.cu).
int estimate_resident(cc_graph_t g, int32_t k, const cc_opts *opts, cc_out *out);
void graph_set_max_ctas(cc_graph_t g, int ctas);
// Sample choice with caller-provided device buffers (no allocation).
int choose_sample_ws(int64_t n, int k, uint64_t seed, int32_t *host_out, void *cand,
                     unsigned *count, int32_t *dout, cudaStream_t st);
size_t sample_candidate_bytes();


}  // namespace ccg
