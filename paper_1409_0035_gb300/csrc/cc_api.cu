// C ABI and host runtime: graph residency, workspace, the traversal passes
// and the estimator pipeline (section 3, Algorithm 1: a pivot/sum pass over
// all k sources, then the hybrid pass when eq. (4) needs per-node L(v)).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "cc_internal.h"
#include "estimate.h"
#include "graph_gpu.h"
#include "nodew.h"
#include "reach.h"
#include "sssp.h"

using namespace ccg;

namespace {

constexpr uint64_t kTimeoutNs = 10ull * 1000 * 1000 * 1000;  // 10 s per wait
// Words per node of the reachability groups (64 sources each; default of
// CC_PARAM_REACH_WORDS).  Directed R-MAT 20 kept whole, k = 64, outbound /
// inbound: 2 words 156 / 154 ms, 4 words 101 / 94 ms, 8 words 85 / 81 ms,
// 16 words 96 / 92 ms (fewer groups and barriers against less pruning).
constexpr int kReachDefaultW = 8;

// Bucket width of the shortest-path rounds in mean arc lengths (default of
// CC_PARAM_SSSP_DELTA).  Measured on the road-like graph (3.9 M nodes, 32
// sources, lengths round(1e3 len)+1 and round(1e6 len)+1): 1 -> 409 / 979
// ms (every bucket a round of its own), 6 -> 245 / 260 ms, 48 -> 211 / 212
// ms, 96 -> 210 / 211 ms, 360 -> 214 ms, 730 -> 223 ms (relaxations per
// node and source 2.65 at small widths, 3.3 at the largest; 8.7 without
// buckets, 391 / 435 ms).
constexpr double kDeltaMult = 96.0;
constexpr double kMaxHistBytes = 4.0 * (1ull << 30);  // distance histogram cap

// Bumped whenever a device buffer is (re)allocated or freed: a captured
// estimate graph holds raw pointers and is valid only while it is unchanged.
std::atomic<uint64_t> g_alloc_gen{1};

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    int ensure(size_t bytes)
    {
        if (bytes <= cap) return CC_OK;
        g_alloc_gen.fetch_add(1);
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            return CC_ERR_OOM;
        }
        cap = bytes;
        return CC_OK;
    }
    void release()
    {
        if (p) g_alloc_gen.fetch_add(1);
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Degree classes of one CSR for the bottom-up scan.
struct Classes {
    DevBuf L, M, H, Hn, Hb, T, Tadj;
    int64_t nL = 0, nM = 0, nH = 0, nHch = 0, nT = 0;
};

// Inline adjacency of the tiny nodes (degree <= kTinyMaxDeg): their
// neighbours as one int4, -1 where the row is shorter.
__global__ void k_tiny_adj(const int32_t *T, int64_t nT, const int64_t *rp, const int32_t *col,
                           int4 *adj)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nT;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = T[t];
        const int64_t b = rp[v], d = rp[v + 1] - b;
        int4 a = make_int4(-1, -1, -1, -1);
        if (d > 0) a.x = col[b];
        if (d > 1) a.y = col[b + 1];
        if (d > 2) a.z = col[b + 2];
        if (d > 3) a.w = col[b + 3];
        adj[t] = a;
    }
}

struct DevCSR {
    DevBuf rp, col, w;
    Classes cls;
};

// Row i of the renumbered CSR is row perm[i] of (rp, col, w) with its
// entries renumbered through iperm (same order).  A warp per row.
__global__ void k_relabel_rows(int64_t n, const int32_t *perm, const int32_t *iperm,
                               const int64_t *rp, const int32_t *col, const uint32_t *w,
                               const int64_t *nrp, int32_t *ncol, uint32_t *nw)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < n; i += nwp) {
        const int32_t v = perm[i];
        const int64_t b = rp[v], d = rp[v + 1] - b, o = nrp[i];
        for (int64_t e = lane; e < d; e += 32) {
            ncol[o + e] = iperm[col[b + e]];
            nw[o + e] = w[b + e];
        }
    }
}

__global__ void k_map_ids(const int32_t *in, int k, const int32_t *map, int32_t *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) out[i] = map[in[i]];
}

// Breadth-first order of the nodes (from node 0, then from each node not
// reached yet): order[i] = the node numbered i.
void bfs_order(int64_t n, const int64_t *rp, const int32_t *col, std::vector<int32_t> &order)
{
    order.clear();
    order.reserve((size_t)n);
    std::vector<uint8_t> seen((size_t)n, 0);
    for (int64_t s0 = 0; s0 < n; ++s0) {
        if (seen[(size_t)s0]) continue;
        seen[(size_t)s0] = 1;
        size_t head = order.size();
        order.push_back((int32_t)s0);
        while (head < order.size()) {
            const int32_t u = order[head++];
            for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
                const int32_t v = col[e];
                if (!seen[(size_t)v]) {
                    seen[(size_t)v] = 1;
                    order.push_back(v);
                }
            }
        }
    }
}

}  // namespace

struct cc_graph {
    int64_t n = 0, arcs = 0;
    bool directed = false, weighted = false;
    DevCSR fw, rv;
    // Undirected graphs with arc lengths: the shortest-path rounds run on
    // lw, the CSR renumbered in breadth-first order (lw_perm: internal ->
    // node id, lw_iperm: node id -> internal; lw_src: a chunk's sources
    // renumbered), so that the nodes a round touches together sit together
    // in memory; their distance rows are read back through lw_iperm.
    DevCSR lw;
    DevBuf lw_perm, lw_iperm, lw_src;
    bool has_lw = false;
    // workspace
    DevBuf vis, F0, F1, nxt, Q0, Q1, T, tflag, sidx, sum2, pivot, delta, lc2, Lmask, hp,
        dcc, hist, TN, TS, Ssamp, maxd, sources, npartial, ctl, shat, clo, hyb, ssum,
        distF, distR, mask, best, dmax, errflag, AL0, AL1, ACH0, ACH1, fstamp, AT0, AT1, ATa0,
        ATa1, band, bflag, gate2, hc2, sp_far0, sp_far1, sp_far2, sp_nst, sp_fst;
    // error estimate of the hybrid (SqErrEst): squared errors, fallback
    // distances, per-node flags, farthest-sample table, staged output
    DevBuf hcse, fdist, sqflag, istar, sqe;
    // adaptive hybrid: one eps's estimate and error, the best so far, choice
    DevBuf ad_est, ad_sq, ad_best, ad_bsq, ad_clo, ad_choice;
    DevBuf pt_clo1, pt_est2, pt_clo2, pt_clo0;  // estimator tables of the finalisation
    // node weights (section 5) and the node-weighted pipeline: sampler
    // scratch, threshold, adjusted weights, sums, histogram, tails, outputs
    DevBuf beta, nw_keys, nw_tk, nw_vals, nw_tv, nw_pre, nw_flags, nw_tau, nw_pick, nw_mu,
        nw_bsrc, nw_msum, nw_wsum, nw_S, nw_hist, nw_TS, nw_lc, nw_out;
    uint64_t beta_total = 0;
    bool has_beta = false;
    // outbound / inbound reachability samples: order, per-node state, queues
    DevBuf rc_order, rc_rank, rc_cnt, rc_extra, rc_dsum, rc_T, rc_qstamp, rc_vis, rc_F, rc_nxt,
        rc_lev, rc_Q0, rc_Q1, rc_TL, rc_out;
    bool sq = false;       // the current cc_estimate call wants SqErrEst
    int64_t D1 = 0;        // levels (largest distance) of the last first pass
    int cw = 32;           // sources per chunk of the last chunked first pass
    bool resident = false; // its distance rows are all kept (chunk c at c * n * cw)
    int64_t dist_max = 0;  // largest distance seen by the last estimate
    int alpha = 0;  // traversal tuning (0: default_alpha)
    bool band_off = false;  // CC_PARAM_HYBRID_ONE_PASS = 0: always two passes
    int64_t sssp_delta = 0;  // CC_PARAM_SSSP_DELTA (0: kDeltaMult x mean length, < 0: off)
    uint32_t band_a = 0, band_b = 0;  // eps the last first pass classified for (0: none)
    int reach_words = 0;     // CC_PARAM_REACH_WORDS (0: kReachDefaultW)
    double w_mean = 0.0;     // mean arc length (weighted graphs)
    int max_ctas = 0;    // cap on the CTAs of each launch (0: whole GPU)
    bool borrowed = false;  // CSR buffers belong to another handle
    int hist_cap = 0;
    Ctl last{};
    // Traversal launches of the last API call: count, device time (CUDA
    // events on the launching stream) and modelled algorithmic bytes.
    int call_launches = 0, call_kernels = 0;
    double call_ms = 0.0, call_bytes = 0.0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // Traversal passes queued without waiting (slot 0: first pass, slot 1:
    // second pass): their control blocks land in pinned hctl[slot] and are
    // read once the call synchronises.
    DevBuf ctl2;
    Ctl *hctl = nullptr;
    cudaEvent_t pev[4] = {nullptr, nullptr, nullptr, nullptr};
    int pend = 0, pend_W[2] = {0, 0};
    uint32_t pend_red[2] = {0, 0};
    // Repeated bit-packed estimates with the same arguments replay one CUDA
    // graph of the whole call (every kernel, memset and control-block copy
    // between the sample upload and the output copies): the call before
    // sizes the buffers, the next one captures.  key: the arguments and
    // buffer generation it was captured for; the queued-pass bookkeeping
    // the capture left is restored on each replay.
    struct EstGraph {
        cudaGraphExec_t exec = nullptr;
        cudaStream_t cap = nullptr;
        std::vector<uint64_t> key, seen, failed;
        bool off = false;      // CC_PARAM_ESTIMATE_GRAPH = 0
        int replayed = 0;      // the last call replayed exec
        int pend = 0, pend_W[2] = {0, 0}, kernels = 0;
        uint32_t pend_red[2] = {0, 0};
    } eg;
};

namespace {

#define CK(x)                                                   \
    do {                                                        \
        cudaError_t e_ = (x);                                   \
        if (e_ != cudaSuccess) {                                \
            note_cuda_error(e_, __FILE__, __LINE__);            \
            cudaGetLastError();                                 \
            return CC_ERR_CUDA;                                 \
        }                                                       \
    } while (0)
#define RC(x)                      \
    do {                           \
        int r_ = (x);              \
        if (r_ != CC_OK) return r_; \
    } while (0)

int upload(DevBuf &b, const void *src, size_t bytes)
{
    RC(b.ensure(bytes));
    if (bytes) CK(cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice));
    return CC_OK;
}

int build_classes(const std::vector<int64_t> &rp, int64_t n, Classes &c, const int64_t *drp,
                  const int32_t *dcol)
{
    // Tiny, light and medium nodes are ordered by degree (stable counting
    // sort, ties by id).  A warp scans W-lane groups of nodes in lock step,
    // so equal degrees keep its lanes busy for the same number of steps; and
    // warps take every nwarps-th entry of a list, so a sorted list hands
    // every warp about the same number of CSR entries.  Tiny nodes (degree
    // <= kTinyMaxDeg) carry their neighbours inline (one int4), which takes
    // two dependent loads out of their scan.
    std::vector<int64_t> start(kMediumMaxDeg + 2, 0);
    for (int64_t v = 0; v < n; ++v) {
        const int64_t d = rp[v + 1] - rp[v];
        if (d <= kMediumMaxDeg) start[d + 1] += 1;
    }
    for (int d = 0; d <= kMediumMaxDeg; ++d) start[d + 1] += start[d];
    const int64_t ntiny = start[kTinyMaxDeg + 1];
    const int64_t nlight = start[kLightMaxDeg + 1];
    std::vector<int32_t> T((size_t)ntiny), L((size_t)(nlight - ntiny)),
        M((size_t)(start[kMediumMaxDeg + 1] - nlight)), H, Hn;
    std::vector<int64_t> Hb;
    for (int64_t v = 0; v < n; ++v) {
        const int64_t d = rp[v + 1] - rp[v];
        if (d <= kTinyMaxDeg) T[(size_t)start[d]++] = (int32_t)v;
        else if (d <= kLightMaxDeg) L[(size_t)(start[d]++ - ntiny)] = (int32_t)v;
        else if (d <= kMediumMaxDeg) M[(size_t)(start[d]++ - nlight)] = (int32_t)v;
        else {
            H.push_back((int32_t)v);
            for (int64_t b = rp[v]; b < rp[v + 1]; b += kChunk) {
                Hn.push_back((int32_t)v);
                Hb.push_back(b);
            }
        }
    }
    c.nL = (int64_t)L.size(); c.nM = (int64_t)M.size(); c.nH = (int64_t)H.size();
    c.nHch = (int64_t)Hn.size();
    c.nT = (int64_t)T.size();
    RC(upload(c.T, T.data(), T.size() * 4));
    RC(c.Tadj.ensure((size_t)std::max<int64_t>(c.nT, 1) * 16));
    if (c.nT > 0) {
        const int64_t g = std::min<int64_t>((c.nT + 255) / 256, 152 * 32);
        k_tiny_adj<<<(int)g, 256>>>(c.T.as<int32_t>(), c.nT, drp, dcol, c.Tadj.as<int4>());
        CK(cudaGetLastError());
        CK(cudaDeviceSynchronize());  // estimates may run on other streams
    }
    RC(upload(c.L, L.data(), L.size() * 4));
    RC(upload(c.M, M.data(), M.size() * 4));
    RC(upload(c.H, H.data(), H.size() * 4));
    RC(upload(c.Hn, Hn.data(), Hn.size() * 4));
    RC(upload(c.Hb, Hb.data(), Hb.size() * 8));
    return CC_OK;
}

int pow2_words(int k)
{
    const int need = (k + 63) / 64;
    int W = 1;
    while (W < need) W <<= 1;
    return W;
}

int ensure_state(cc_graph *g, int W)
{
    const int64_t n = g->n;
    const size_t nw = (size_t)n * W * 8;
    RC(g->vis.ensure(nw));
    RC(g->F0.ensure(nw));
    RC(g->F1.ensure(nw));
    RC(g->nxt.ensure(nw));
    RC(g->Q0.ensure(n * 4));
    RC(g->Q1.ensure(n * 4));
    RC(g->T.ensure(n * 4));
    RC(g->AL0.ensure(n * 4));
    RC(g->AL1.ensure(n * 4));
    const int64_t nch = std::max(g->fw.cls.nHch, g->rv.cls.nHch);
    RC(g->ACH0.ensure((size_t)nch * 4));
    RC(g->ACH1.ensure((size_t)nch * 4));
    const int64_t nt = std::max<int64_t>(std::max(g->fw.cls.nT, g->rv.cls.nT), 1);
    RC(g->AT0.ensure((size_t)nt * 4));
    RC(g->AT1.ensure((size_t)nt * 4));
    RC(g->ATa0.ensure((size_t)nt * 16));
    RC(g->ATa1.ensure((size_t)nt * 16));
    RC(g->fstamp.ensure(n * 4));
    RC(g->tflag.ensure(n * 4));
    RC(g->sidx.ensure(n * 4));
    RC(g->sum2.ensure(n * 16));
    RC(g->ctl.ensure(sizeof(Ctl)));
    return CC_OK;
}

// Pass over `push` (top-down, arcs leaving a node) and `pull` (bottom-up,
// arcs entering a node): the same CSR for undirected graphs; G and G^T for
// a forward pass on a directed graph, G^T and G for a reverse pass.
BfsJob base_job(cc_graph *g, int W, const DevCSR &push, const DevCSR &pull)
{
    const DevCSR &csr = pull;
    BfsJob j;
    std::memset(&j, 0, sizeof(j));
    j.n = g->n;
    j.arcs = g->arcs;
    j.rp = push.rp.as<int64_t>();
    j.col = push.col.as<int32_t>();
    j.tHn = push.cls.Hn.as<int32_t>();
    j.tHb = push.cls.Hb.as<int64_t>();
    j.ntH = push.cls.nHch;
    j.prp = pull.rp.as<int64_t>();
    j.pcol = pull.col.as<int32_t>();
    j.Llist = csr.cls.L.as<int32_t>();
    j.Mlist = csr.cls.M.as<int32_t>();
    j.Hlist = csr.cls.H.as<int32_t>();
    j.nL = csr.cls.nL;
    j.nM = csr.cls.nM;
    j.nH = csr.cls.nH;
    j.Hch_node = csr.cls.Hn.as<int32_t>();
    j.Hch_begin = csr.cls.Hb.as<int64_t>();
    j.nHch = csr.cls.nHch;
    j.vis = g->vis.as<uint64_t>();
    j.F0 = g->F0.as<uint64_t>();
    j.F1 = g->F1.as<uint64_t>();
    j.nxt = g->nxt.as<uint64_t>();
    j.Q0 = g->Q0.as<int32_t>();
    j.Q1 = g->Q1.as<int32_t>();
    j.T = g->T.as<int32_t>();
    j.AL0 = g->AL0.as<int32_t>();
    j.AL1 = g->AL1.as<int32_t>();
    j.ACH0 = g->ACH0.as<int32_t>();
    j.ACH1 = g->ACH1.as<int32_t>();
    j.Tlist = csr.cls.T.as<int32_t>();
    j.Tadj = csr.cls.Tadj.as<int4>();
    j.nT = csr.cls.nT;
    j.AT0 = g->AT0.as<int32_t>();
    j.AT1 = g->AT1.as<int32_t>();
    j.ATa0 = g->ATa0.as<int4>();
    j.ATa1 = g->ATa1.as<int4>();
    j.fstamp = g->fstamp.as<uint32_t>();
    j.tflag = g->tflag.as<unsigned>();
    j.sidx = g->sidx.as<int32_t>();
    j.sum2 = g->sum2.as<uint64_t>();
    j.ctl = g->ctl.as<Ctl>();
    j.timeout_ns = kTimeoutNs;
    j.alpha = g->alpha ? g->alpha : default_alpha(W, j.n, j.arcs);
    j.max_ctas = g->max_ctas;
    return j;
}

void reset_timing(cc_graph *g)
{
    g->call_launches = 0;
    g->call_kernels = 0;
    g->call_ms = 0.0;
    g->call_bytes = 0.0;
}

// Algorithmic bytes of one traversal pass (the roofline model of the design
// notes): every frontier word gathered (8 B) with its CSR entry (4 B, one per
// W words), three word arrays (visited, frontier in, frontier out) per node
// and level, the row offsets of top-down levels and R bytes of per-node
// results.
double pass_bytes(const Ctl &c, int64_t n, int W, uint32_t red)
{
    const double words = (double)c.words;
    const double R = (red & RED_LC) ? 16.0 : ((red & RED_PIVOT) ? 24.0 : 16.0);
    return words * 8.0 + words / W * 4.0 + (double)c.levels * n * 8.0 * W * 3.0 +
           (double)c.td_levels * (n + 1) * 8.0 + (double)n * R;
}

// Queue one pass in slot 0 or 1 without waiting: its control block (slot
// 1: g->ctl2) is cleared before and copied to the pinned g->hctl[slot]
// after, between two events.  settle_passes reads them.
int queue_pass(cc_graph *g, int slot, int W, BfsJob j, cudaStream_t st)
{
    if (!g->hctl) CK(cudaMallocHost(&g->hctl, 2 * sizeof(Ctl)));
    for (cudaEvent_t &e : g->pev)
        if (!e) CK(cudaEventCreate(&e));
    if (slot == 1) RC(g->ctl2.ensure(sizeof(Ctl)));
    Ctl *dctl = slot == 0 ? g->ctl.as<Ctl>() : g->ctl2.as<Ctl>();
    j.ctl = dctl;
    CK(cudaMemsetAsync(dctl, 0, sizeof(Ctl), st));
    // Inside a stream capture, a timing record must be an external one.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs));
    const unsigned rf = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    CK(cudaEventRecordWithFlags(g->pev[2 * slot], st, rf));
    RC(launch_msbfs(W, j, st, nullptr));
    CK(cudaEventRecordWithFlags(g->pev[2 * slot + 1], st, rf));
    CK(cudaMemcpyAsync(&g->hctl[slot], dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    g->pend |= 1 << slot;
    g->pend_W[slot] = W;
    g->pend_red[slot] = j.red;
    g->call_kernels += 1;
    return CC_OK;
}

// After the stream has been synchronised: account the queued passes (a
// second pass whose gate skipped it left a zero control block) and copy the
// last one that ran to g->last.  Returns the first negative error code.
int settle_passes(cc_graph *g)
{
    int rc = CC_OK;
    for (int slot = 0; slot < 2; ++slot) {
        if (!(g->pend & (1 << slot))) continue;
        const Ctl &c = g->hctl[slot];
        if (slot == 1 && c.levels == 0 && c.words == 0) continue;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, g->pev[2 * slot], g->pev[2 * slot + 1]));
        g->last = c;
        g->last.edges = c.words / (unsigned long long)g->pend_W[slot];
        g->call_launches += 1;
        g->call_ms += ms;
        g->call_bytes += pass_bytes(c, g->n, g->pend_W[slot], g->pend_red[slot]);
        if (c.err < 0 && rc == CC_OK) rc = c.err;
    }
    g->pend = 0;
    return rc;
}

// Launch one pass and wait for it; copies the control block to g->last.
int run_pass(cc_graph *g, int W, const BfsJob &j, cudaStream_t st)
{
    RC(queue_pass(g, 0, W, j, st));
    CK(cudaStreamSynchronize(st));
    return settle_passes(g);
}

// Ids in range and distinct, from a sorted copy of the k ids: the check runs
// on every call, so it takes no per-node host array.
int validate_sample(const cc_graph *g, const int32_t *sample, int32_t k)
{
    if (!sample || k < 1 || k > CC_MAX_K || k > g->n) return CC_ERR_ARG;
    std::vector<int32_t> s(sample, sample + k);
    std::sort(s.begin(), s.end());
    if (s[0] < 0 || s[(size_t)k - 1] >= g->n) return CC_ERR_ARG;
    for (int i = 1; i < k; ++i)
        if (s[(size_t)i] == s[(size_t)i - 1]) return CC_ERR_ARG;
    return CC_OK;
}

// G^T of a directed graph built on the device into g->rv.
int adopt_device_reverse(cc_graph *g, DeviceCSR &d)
{
    g->rv.rp.p = d.rp;
    g->rv.rp.cap = (size_t)(d.n + 1) * 8;
    g->rv.col.p = d.col;
    g->rv.col.cap = (size_t)std::max<int64_t>(d.arcs, 1) * 4;
    if (d.w) {
        g->rv.w.p = d.w;
        g->rv.w.cap = (size_t)std::max<int64_t>(d.arcs, 1) * 4;
    }
    d.rp = d.col = d.w = nullptr;
    return build_classes(d.rp_host, d.n, g->rv.cls, g->rv.rp.as<int64_t>(),
                         g->rv.col.as<int32_t>());
}

// Take ownership of a CSR built on the device.
int adopt_device_csr(cc_graph *g, DeviceCSR &d)
{
    g->n = d.n;
    g->arcs = d.arcs;
    g->weighted = d.w != nullptr;
    g->fw.rp.p = d.rp;
    g->fw.rp.cap = (size_t)(d.n + 1) * 8;
    g->fw.col.p = d.col;
    g->fw.col.cap = (size_t)std::max<int64_t>(d.arcs, 1) * 4;
    if (d.w) {
        g->fw.w.p = d.w;
        g->fw.w.cap = (size_t)std::max<int64_t>(d.arcs, 1) * 4;
    }
    d.rp = d.col = d.w = nullptr;
    return build_classes(d.rp_host, d.n, g->fw.cls, g->fw.rp.as<int64_t>(),
                         g->fw.col.as<int32_t>());
}

// The breadth-first renumbering of an undirected graph with arc lengths
// (cc_graph::lw), from the host copy of its row offsets.
int build_locality(cc_graph *g, const std::vector<int64_t> &rp)
{
    const int64_t n = g->n, arcs = g->arcs;
    std::vector<int32_t> col((size_t)arcs);
    if (arcs) CK(cudaMemcpy(col.data(), g->fw.col.p, (size_t)arcs * 4, cudaMemcpyDeviceToHost));
    std::vector<int32_t> perm, iperm((size_t)n);
    bfs_order(n, rp.data(), col.data(), perm);
    for (int64_t i = 0; i < n; ++i) iperm[(size_t)perm[(size_t)i]] = (int32_t)i;
    std::vector<int64_t> nrp((size_t)n + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        const int32_t v = perm[(size_t)i];
        nrp[(size_t)i + 1] = nrp[(size_t)i] + (rp[(size_t)v + 1] - rp[(size_t)v]);
    }
    RC(upload(g->lw_perm, perm.data(), (size_t)n * 4));
    RC(upload(g->lw_iperm, iperm.data(), (size_t)n * 4));
    RC(upload(g->lw.rp, nrp.data(), ((size_t)n + 1) * 8));
    RC(g->lw.col.ensure((size_t)std::max<int64_t>(arcs, 1) * 4));
    RC(g->lw.w.ensure((size_t)std::max<int64_t>(arcs, 1) * 4));
    const int64_t grid = std::min<int64_t>((n * 32 + 255) / 256, 152 * 32);
    k_relabel_rows<<<(int)std::max<int64_t>(grid, 1), 256>>>(
        n, g->lw_perm.as<int32_t>(), g->lw_iperm.as<int32_t>(), g->fw.rp.as<int64_t>(),
        g->fw.col.as<int32_t>(), g->fw.w.as<uint32_t>(), g->lw.rp.as<int64_t>(),
        g->lw.col.as<int32_t>(), g->lw.w.as<uint32_t>());
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());  // estimates may run on other streams
    g->has_lw = true;
    return CC_OK;
}

void free_graph(cc_graph *g)
{
    if (g->borrowed) {  // drop the borrowed CSR pointers unfreed
        DevBuf *csr[] = {&g->fw.rp, &g->fw.col, &g->fw.w, &g->lw.rp, &g->lw.col, &g->lw.w,
                         &g->lw_perm, &g->lw_iperm, &g->fw.cls.L, &g->fw.cls.M,
                         &g->fw.cls.H, &g->fw.cls.Hn, &g->fw.cls.Hb, &g->fw.cls.T, &g->fw.cls.Tadj,
                     &g->rv.rp, &g->rv.col,
                         &g->rv.w, &g->rv.cls.L, &g->rv.cls.M, &g->rv.cls.H, &g->rv.cls.Hn,
                         &g->rv.cls.Hb, &g->rv.cls.T, &g->rv.cls.Tadj};
        for (DevBuf *b : csr) { b->p = nullptr; b->cap = 0; }
    }
    DevBuf *all[] = {&g->fw.rp, &g->fw.col, &g->fw.w, &g->lw.rp, &g->lw.col, &g->lw.w,
                     &g->lw_perm, &g->lw_iperm, &g->lw_src, &g->fw.cls.L, &g->fw.cls.M,
                     &g->fw.cls.H, &g->fw.cls.Hn, &g->fw.cls.Hb, &g->fw.cls.T, &g->fw.cls.Tadj,
                     &g->rv.rp, &g->rv.col,
                     &g->rv.w, &g->rv.cls.L, &g->rv.cls.M, &g->rv.cls.H, &g->rv.cls.Hn,
                     &g->rv.cls.Hb, &g->rv.cls.T, &g->rv.cls.Tadj, &g->vis, &g->F0, &g->F1, &g->nxt, &g->Q0, &g->Q1,
                     &g->T, &g->tflag, &g->sidx, &g->sum2, &g->pivot, &g->delta, &g->lc2,
                     &g->Lmask, &g->hp, &g->dcc, &g->hist, &g->TN, &g->TS, &g->Ssamp,
                     &g->maxd, &g->sources, &g->npartial, &g->ctl, &g->shat, &g->clo,
                     &g->hyb, &g->ssum, &g->distF, &g->distR, &g->mask, &g->best,
                     &g->dmax, &g->errflag, &g->AL0, &g->AL1, &g->ACH0, &g->ACH1, &g->fstamp, &g->AT0, &g->AT1,
                     &g->ATa0, &g->ATa1, &g->band, &g->bflag, &g->gate2, &g->hc2, &g->sp_far0, &g->sp_far1, &g->sp_far2, &g->sp_nst, &g->sp_fst,
                     &g->hcse, &g->fdist, &g->sqflag, &g->istar, &g->sqe,
                     &g->ad_est, &g->ad_sq, &g->ad_best, &g->ad_bsq, &g->ad_clo, &g->ad_choice,
                     &g->pt_clo1, &g->pt_est2, &g->pt_clo2, &g->pt_clo0,
                     &g->beta, &g->nw_keys, &g->nw_tk, &g->nw_vals, &g->nw_tv, &g->nw_pre,
                     &g->nw_flags, &g->nw_tau, &g->nw_pick, &g->nw_mu, &g->nw_bsrc,
                     &g->nw_msum, &g->nw_wsum, &g->nw_S, &g->nw_hist, &g->nw_TS, &g->nw_lc,
                     &g->nw_out, &g->rc_order, &g->rc_rank, &g->rc_cnt, &g->rc_extra,
                     &g->rc_dsum, &g->rc_T, &g->rc_qstamp, &g->rc_vis, &g->rc_F, &g->rc_nxt,
                     &g->rc_lev, &g->rc_Q0, &g->rc_Q1, &g->rc_TL, &g->rc_out};
    for (DevBuf *b : all) b->release();
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    g->ev0 = g->ev1 = nullptr;
    for (cudaEvent_t &e : g->pev)
        if (e) { cudaEventDestroy(e); e = nullptr; }
    if (g->hctl) { cudaFreeHost(g->hctl); g->hctl = nullptr; }
    if (g->eg.exec) { cudaGraphExecDestroy(g->eg.exec); g->eg.exec = nullptr; }
    if (g->eg.cap) { cudaStreamDestroy(g->eg.cap); g->eg.cap = nullptr; }
}


// Unweighted undirected graphs: one bit-packed multi-source pass for sums,
// pivots, Delta, delta_cc and the per-level histogram, and a second pass
// with the L(v) masks only when some node's L(v) misses a sampled node.
// Buffers and the farthest-sample table of the error estimate.
int prepare_sq(cc_graph *g, int k, cudaStream_t st)
{
    const int64_t n = g->n;
    RC(g->hcse.ensure((size_t)n * 16));
    RC(g->fdist.ensure((size_t)n * 4));
    RC(g->sqflag.ensure((size_t)n));
    RC(g->istar.ensure((size_t)k * 4));
    CK(cudaMemsetAsync(g->hcse.p, 0, (size_t)n * 16, st));
    run_istar(g->dcc.as<uint32_t>(), k, g->istar.as<int32_t>(), st);
    g->call_kernels += 1;
    return CC_OK;
}

// First pass of the bit-packed path: sums, pivots, Delta, delta_cc, the
// per-source level histogram and the exact S of the sampled nodes.
// With eps_a > 0 the pass also classifies each arriving bit for the hybrid
// of eps = eps_a / eps_b (RED_BAND), so that no second pass is needed.
int bfs_pass1(cc_graph *g, int k, cudaStream_t st, uint32_t eps_a = 0, uint32_t eps_b = 0)
{
    const int64_t n = g->n;
    const int W = pow2_words(k);
    RC(ensure_state(g, W));
    if (g->hist_cap == 0) g->hist_cap = (int)std::min<int64_t>(n + 1, 4096);
    BfsJob j = base_job(g, W, g->fw, g->fw);
    j.k = k;
    j.sources = g->sources.as<int32_t>();
    j.red = RED_SUM | RED_PIVOT | RED_DCC | RED_HIST;
    g->band_a = eps_a;
    g->band_b = eps_b;
    if (eps_a > 0) {
        RC(g->band.ensure((size_t)n * 64 * W));
        RC(g->bflag.ensure((size_t)n));
        RC(g->hc2.ensure(n * 16));
        j.red |= RED_BAND;
        j.band = g->band.as<uint8_t>();
        j.bflag = g->bflag.as<uint8_t>();
        j.lc2 = g->hc2.as<uint64_t>();  // the sums over HC(v) settled on arrival
        j.eps_a = eps_a;
        j.eps_b = eps_b;
    }
    j.pivot = g->pivot.as<int32_t>();
    j.delta = g->delta.as<uint32_t>();
    j.dcc = g->dcc.as<uint32_t>();
    j.dcc_k = k;
    // Queued without waiting: the kernels after it read the level count
    // from the control block on the device, and check_pass1 looks at the
    // outcome once the call has synchronised.
    RC(g->hist.ensure((size_t)g->hist_cap * k * 4));
    j.hist = g->hist.as<uint32_t>();
    j.hist_cap = g->hist_cap;
    CK(cudaMemsetAsync(g->sum2.p, 0, n * 16, st));
    CK(cudaMemsetAsync(g->hist.p, 0, (size_t)g->hist_cap * k * 4, st));
    CK(cudaMemsetAsync(g->dcc.p, 0, (size_t)k * k * 4, st));
    RC(queue_pass(g, 0, W, j, st));
    run_S_sampled(g->hist.as<uint32_t>(), DevCount{&g->ctl.as<Ctl>()->levels, 0}, k,
                  g->dcc.as<uint32_t>(), g->Ssamp.as<uint64_t>(), st);
    g->call_kernels += 1;
    return CC_OK;
}

// Outcome of the queued first pass, after the stream synchronised:
// CC_ERR_DISCONNECTED when some node was never reached, 1 when the level
// histogram was too short (the caller grows it and runs the call again).
int check_pass1(cc_graph *g, bool hybrid, int k)
{
    const Ctl &c = g->hctl[0];
    if (c.err == 1) {
        if (g->hist_cap > g->n) return CC_ERR_TOO_LARGE;
        g->hist_cap = (int)std::min<int64_t>(g->n + 1, (int64_t)g->hist_cap * 4);
        return 1;
    }
    if (c.ninc_final != 0) return CC_ERR_DISCONNECTED;
    g->dist_max = c.levels;
    g->D1 = c.levels;
    // Sums of squared levels (LCsumSq, the squared errors) stay in 64 bits.
    if (hybrid && (double)c.levels * (double)c.levels * (double)k >= 1.8e19)
        return CC_ERR_TOO_LARGE;
    return CC_OK;
}

// The hybrid part of the bit-packed path for eps = a/b, after bfs_pass1:
// H statistics from the histogram tails, thresholds, L-masks and, where
// needed, the second pass.
int bfs_hybrid(cc_graph *g, int k, uint32_t a, uint32_t b, cudaStream_t st, bool band = false)
{
    const int64_t n = g->n;
    const int W = pow2_words(k);
    // The level count D of the first pass stays on the device; the tail
    // tables have hist_cap >= D + 1 entries per source.
    const DevCount D{&g->ctl.as<Ctl>()->levels, 0};
    const int64_t stride = g->hist_cap;
    RC(g->TN.ensure((size_t)k * stride * 8));
    RC(g->TS.ensure((size_t)k * stride * 8));
    RC(g->maxd.ensure((size_t)k * 4));
    RC(g->hp.ensure((size_t)n * sizeof(HybPrep)));
    RC(g->npartial.ensure(8));
    CK(cudaMemsetAsync(g->npartial.p, 0, 8, st));
    run_tail(g->hist.as<uint32_t>(), D, stride, k, g->TN.as<uint64_t>(), g->TS.as<uint64_t>(),
             st);
    run_maxdelta(g->dcc.as<uint32_t>(), k, g->maxd.as<uint32_t>(), st);
    SqPrep sq{nullptr};
    if (g->sq) {
        RC(prepare_sq(g, k, st));
        sq.flag = g->sqflag.as<uint8_t>();
    }
    run_hyb_prep(3, n, k, D, stride, a, b, g->sidx.as<int32_t>(),
                 g->pivot.as<int32_t>(), g->delta.as<uint32_t>(), g->dcc.as<uint32_t>(),
                 g->maxd.as<uint32_t>(), g->TN.as<uint64_t>(), g->TS.as<uint64_t>(),
                 g->hp.as<HybPrep>(), g->npartial.as<unsigned>(), sq, st);
    g->call_kernels += 3;
    RC(g->lc2.ensure(n * 16));
    // The second pass gathers LCsum for nodes whose L(v) misses a sampled
    // node and, for the error estimate, the squared errors over HC(v) or
    // the distance to the farthest sample where HC(v) is empty.  It is
    // queued regardless and exits at once (like the L-mask kernel) when the
    // preparation counted no such node.  After a first pass that
    // classified on arrival, LCsum is complete once the deferred bits are
    // resolved, and the second pass runs only if a band offset overflowed.
    const unsigned *gate = g->npartial.as<unsigned>();
    if (band) {
        RC(g->gate2.ensure(8));
        run_band_resolve(n, k, 64 * W, g->sidx.as<int32_t>(), g->pivot.as<int32_t>(),
                         g->delta.as<uint32_t>(), g->dcc.as<uint32_t>(), g->hp.as<HybPrep>(),
                         g->bflag.as<uint8_t>(), g->band.as<uint8_t>(),
                         g->sum2.as<uint64_t>(), g->hc2.as<uint64_t>(), g->lc2.as<uint64_t>(),
                         &g->ctl.as<Ctl>()->band_ovf, g->gate2.as<unsigned>(),
                         g->npartial.as<unsigned>(), st);
        g->call_kernels += 1;
        gate = g->gate2.as<unsigned>();
    }
    RC(g->Lmask.ensure((size_t)n * W * 8));
    run_lmask(n, W, k, g->sidx.as<int32_t>(), g->pivot.as<int32_t>(), g->dcc.as<uint32_t>(),
              g->hp.as<HybPrep>(), g->Lmask.as<uint64_t>(), gate, st);
    g->call_kernels += 1;
    BfsJob j2 = base_job(g, W, g->fw, g->fw);
    j2.gate = gate;
    j2.k = k;
    j2.sources = g->sources.as<int32_t>();
    j2.red = RED_LC;
    j2.Lmask = g->Lmask.as<uint64_t>();
    j2.lc2 = g->lc2.as<uint64_t>();
    if (g->sq) {
        j2.red |= RED_SQ;
        j2.pivot = g->pivot.as<int32_t>();
        j2.dcc = g->dcc.as<uint32_t>();
        j2.dcc_k = k;
        j2.sqflag = g->sqflag.as<uint8_t>();
        j2.istar = g->istar.as<int32_t>();
        j2.hcse = g->hcse.as<uint64_t>();
        j2.fdist = g->fdist.as<uint32_t>();
    }
    return queue_pass(g, 1, W, j2, st);
}

// Whether the first pass can classify the hybrid's bits on arrival: the
// plain hybrid (not its error estimate, which needs every sampled node's
// distance) while the band rows (64W bytes per node) fit in a third of the
// free device memory.
bool use_band(cc_graph *g, int k, const cc_opts *opts)
{
    if (!opts->want_hybrid || g->sq || g->band_off) return false;
    const double need = (double)g->n * 64.0 * pow2_words(k);
    if ((double)g->band.cap >= need) return true;  // rows held from an earlier call
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return need <= ((double)free_b + (double)g->band.cap) / 3.0;
}

int estimate_bfs(cc_graph *g, int k, const cc_opts *opts, bool band, cudaStream_t st)
{
    RC(bfs_pass1(g, k, st, band ? opts->eps_num : 0, band ? opts->eps_den : 0));
    if (!opts->want_hybrid) return CC_OK;
    return bfs_hybrid(g, k, opts->eps_num, opts->eps_den, st, band);
}

// One chunk of shortest paths (forward, and reversed for round trips)
// into g->distF / g->distR.  Unit lengths use the bit-packed traversal
// writing levels; arc lengths the delta-stepping kernel.  Sources per
// chunk: with arc lengths 64 (two per lane of a 256-byte row: the rounds,
// whose fixed cost bounds a chunk on graphs of large diameter, are shared
// by twice the sources) or 32; with unit lengths up to 128 (two bit-packed
// words per node) so that fewer, wider traversals fill the rows; always
// while the distance rows (one or two n x cw tables) take at most a third
// of the free device memory.
int chunk_width(cc_graph *g, int64_t k)
{
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return kChunkSrc;
    }
    const double tables = g->directed ? 2.0 : 1.0;
    int cw = g->weighted ? 2 * kChunkSrc : 128;
    while (cw > kChunkSrc && (double)g->n * cw * 4.0 * tables > (double)free_b / 3.0) cw /= 2;
    while (cw > kChunkSrc && cw / 2 >= k) cw /= 2;
    return cw;
}

// Whether `bytes` of rows per table (two tables for round trips) fit in a
// third of the device memory that is free or already held by the rows.
bool rows_fit(cc_graph *g, size_t bytes)
{
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const double tables = g->directed ? 2.0 : 1.0;
    const double avail = (double)free_b + (double)g->distF.cap + (double)g->distR.cap;
    return (double)bytes * tables <= avail / 3.0;
}

// First element of the rows of the chunk starting at source `base`.
size_t chunk_offset(const cc_graph *g, int base)
{
    return g->resident ? (size_t)(base / g->cw) * (size_t)g->n * g->cw : 0;
}

// Bucket width of the shortest-path rounds: kDeltaMult x the mean arc
// length unless set (CC_PARAM_SSSP_DELTA; negative: no buckets).
uint64_t sssp_delta(const cc_graph *g)
{
    if (!g->weighted || g->sssp_delta < 0) return 0;
    if (g->sssp_delta > 0) return (uint64_t)g->sssp_delta;
    return (uint64_t)std::max(1.0, std::round(kDeltaMult * g->w_mean));
}

// off: first element of the chunk's rows in distF / distR.
int run_chunk(cc_graph *g, const int32_t *d_sources, int kc, int cw, cudaStream_t st,
              size_t off)
{
    const int64_t n = g->n;
    if (!g->weighted) {
        const int W = pow2_words(kc);
        RC(ensure_state(g, W));
        // An undirected graph is its own reverse (no separate G^T is kept).
        const DevCSR &gt = g->directed ? g->rv : g->fw;
        for (int dir = 0; dir < (g->directed ? 2 : 1); ++dir) {
            BfsJob j = base_job(g, W, dir ? gt : g->fw, dir ? g->fw : gt);
            j.k = kc;
            j.sources = d_sources;
            j.red = RED_LEVELS;
            j.dist_out = (dir ? g->distR : g->distF).as<uint32_t>() + off;
            j.dist_ld = cw;
            RC(run_pass(g, W, j, st));
            if (g->last.ninc_final != 0) return CC_ERR_DISCONNECTED;
        }
        return CC_OK;
    }
    // Undirected: the breadth-first renumbered CSR, sources renumbered.
    const bool lw = g->has_lw && !g->directed;
    if (lw) {
        RC(g->lw_src.ensure((size_t)kc * 4));
        k_map_ids<<<(kc + 255) / 256, 256, 0, st>>>(d_sources, kc, g->lw_iperm.as<int32_t>(),
                                                     g->lw_src.as<int32_t>());
        CK(cudaGetLastError());
        g->call_kernels += 1;
    }
    for (int dir = 0; dir < (g->directed ? 2 : 1); ++dir) {
        const DevCSR &c = lw ? g->lw : dir ? g->rv : g->fw;
        SsspJob j;
        std::memset(&j, 0, sizeof(j));
        j.n = n;
        j.rp = c.rp.as<int64_t>();
        j.col = c.col.as<int32_t>();
        j.w = g->weighted ? c.w.as<uint32_t>() : nullptr;
        j.kc = kc;
        j.sources = lw ? g->lw_src.as<int32_t>() : d_sources;
        j.dist = (dir ? g->distR : g->distF).as<uint32_t>() + off;
        j.mask = g->mask.as<unsigned long long>();
        j.spl = cw / kChunkSrc;
        j.Q0 = g->Q0.as<int32_t>();
        j.Q1 = g->Q1.as<int32_t>();
        j.delta = sssp_delta(g);
        if (j.delta) {
            RC(g->sp_far0.ensure(n * 4));
            RC(g->sp_far1.ensure(n * 4));
            RC(g->sp_far2.ensure(n * 4));
            RC(g->sp_nst.ensure(n * 4));
            RC(g->sp_fst.ensure(n * 4));
            j.far[0] = g->sp_far0.as<int32_t>();
            j.far[1] = g->sp_far1.as<int32_t>();
            j.far[2] = g->sp_far2.as<int32_t>();
            j.nstamp = g->sp_nst.as<uint32_t>();
            j.fstamp = g->sp_fst.as<uint32_t>();
        }
        j.ctl = g->ctl.as<Ctl>();
        j.timeout_ns = kTimeoutNs;
        j.max_ctas = g->max_ctas;
        if (!g->ev0) {
            CK(cudaEventCreate(&g->ev0));
            CK(cudaEventCreate(&g->ev1));
        }
        CK(cudaMemsetAsync(g->ctl.p, 0, sizeof(Ctl), st));
        CK(cudaEventRecord(g->ev0, st));
        RC(launch_mssp(j, st));
        CK(cudaEventRecord(g->ev1, st));
        CK(cudaMemcpyAsync(&g->last, g->ctl.p, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
        g->call_launches += 1;
        g->call_kernels += 1;
        g->call_ms += ms;
        // relaxations x (row read 4 B + arc 8 B) + the n x 32 rows written once
        g->call_bytes += (double)g->last.words * 12.0 + (double)n * cw * 4.0;
        if (g->last.err < 0) return g->last.err;
    }
    return CC_OK;
}

// Whether the chunk rows of g are indexed by the breadth-first numbering
// (shortest-path rounds on cc_graph::lw).
bool rows_renumbered(const cc_graph *g) { return g->weighted && g->has_lw && !g->directed; }

ReduceJob base_reduce(cc_graph *g, int k, int W)
{
    ReduceJob r;
    std::memset(&r, 0, sizeof(r));
    r.n = g->n;
    r.k = k;
    r.W = W;
    r.distF = g->distF.as<uint32_t>();
    r.distR = g->directed ? g->distR.as<uint32_t>() : nullptr;
    r.row_of = rows_renumbered(g) ? g->lw_iperm.as<int32_t>() : nullptr;
    r.sidx = g->sidx.as<int32_t>();
    r.sum2 = g->sum2.as<uint64_t>();
    r.best = g->best.as<unsigned long long>();
    r.dcc = g->dcc.as<uint32_t>();
    r.S_samp = g->Ssamp.as<unsigned long long>();
    r.dmax = g->dmax.as<unsigned long long>();
    r.err = g->errflag.as<int>();
    return r;
}

// Weighted or directed (round-trip) graphs: the k sources in 32-source
// chunks of shortest paths, each reduced into the same per-node statistics;
// the hybrid needs a second sweep (histogram of distances and L(v) sums).
// First pass of the chunked path (weighted graphs, round trips): 32-source
// chunks of shortest paths reduced into sums, pivots, Delta, delta_cc and
// the exact S of the sampled nodes.
// nw (optional): the node-weighted sums, reduced from the same rows.
int chunked_pass1(cc_graph *g, int k, cudaStream_t st, const NwJob *nw = nullptr)
{
    const int64_t n = g->n;
    const int W = pow2_words(k);
    const int cw = chunk_width(g, k);
    g->cw = cw;
    // Keep every chunk's rows when they fit in a third of the free memory:
    // the hybrid's second sweep (and each eps of the adaptive hybrid) then
    // reduces them again instead of repeating the traversals.
    const int nch = (k + cw - 1) / cw;
    g->resident = nch == 1 || rows_fit(g, (size_t)n * cw * nch * 4);
    const size_t rows = (size_t)n * cw * (g->resident ? nch : 1) * 4;
    RC(g->distF.ensure(rows));
    if (g->directed) RC(g->distR.ensure(rows));
    RC(g->mask.ensure(n * 8));
    RC(g->Q0.ensure(n * 4));
    RC(g->Q1.ensure(n * 4));
    RC(g->best.ensure(n * 8));
    RC(g->dmax.ensure(8));
    RC(g->errflag.ensure(4));
    CK(cudaMemsetAsync(g->sum2.p, 0, n * 16, st));
    CK(cudaMemsetAsync(g->best.p, 0xFF, n * 8, st));
    CK(cudaMemsetAsync(g->dcc.p, 0, (size_t)k * k * 4, st));
    CK(cudaMemsetAsync(g->Ssamp.p, 0, (size_t)k * 8, st));
    CK(cudaMemsetAsync(g->dmax.p, 0, 8, st));
    CK(cudaMemsetAsync(g->errflag.p, 0, 4, st));
    const int32_t *src = g->sources.as<int32_t>();
    ReduceJob r = base_reduce(g, k, W);
    r.ld = cw;
    for (int base = 0; base < k; base += cw) {
        const int kc = std::min(cw, k - base);
        const size_t off = chunk_offset(g, base);
        RC(run_chunk(g, src + base, kc, cw, st, off));
        r.distF = g->distF.as<uint32_t>() + off;
        r.distR = g->directed ? g->distR.as<uint32_t>() + off : nullptr;
        for (int s = 0; s < kc; s += 32) {  // one reduction per 32 columns
            r.base = base + s;
            r.sub = s;
            r.kc = std::min(32, kc - s);
            run_reduce1(r, st);
            g->call_kernels += 1;
            if (nw) {
                NwJob j = *nw;
                j.distF = r.distF;
                j.distR = r.distR;
                j.base = r.base;
                j.sub = s;
                j.kc = r.kc;
                j.ld = cw;
                run_nw_reduce1(j, st);
                g->call_kernels += 1;
            }
        }
    }
    unsigned long long dmax = 0;
    int err = 0;
    CK(cudaMemcpyAsync(&dmax, g->dmax.p, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&err, g->errflag.p, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (err) return err;
    run_unpack_pivot(n, g->best.as<unsigned long long>(), g->pivot.as<int32_t>(),
                     g->delta.as<uint32_t>(), st);
    g->call_kernels += 1;
    g->dist_max = (int64_t)dmax;
    g->D1 = (int64_t)dmax;
    return CC_OK;
}

// The hybrid part of the chunked path for eps = a/b, after chunked_pass1:
// thresholds and L-masks, the chunks again for the distance histogram and
// the L(v) n C sums, then the H statistics from the histogram tails.
int chunked_hybrid(cc_graph *g, int k, uint32_t a, uint32_t b, cudaStream_t st)
{
    const int64_t n = g->n;
    const int W = pow2_words(k);
    const int32_t *src = g->sources.as<int32_t>();
    ReduceJob r = base_reduce(g, k, W);
    const int64_t D = g->D1;
    if ((double)(D + 1) * k * 4.0 > (double)kMaxHistBytes) return CC_ERR_TOO_LARGE;
    // Sums of squared distances (LCsumSq) stay in 64 bits.
    if ((double)D * (double)D * (double)k >= 1.8e19) return CC_ERR_TOO_LARGE;
    RC(g->hist.ensure((size_t)(D + 1) * k * 4));
    RC(g->TN.ensure((size_t)k * (D + 1) * 8));
    RC(g->TS.ensure((size_t)k * (D + 1) * 8));
    RC(g->maxd.ensure((size_t)k * 4));
    RC(g->hp.ensure((size_t)n * sizeof(HybPrep)));
    RC(g->npartial.ensure(8));
    RC(g->Lmask.ensure((size_t)n * W * 8));
    RC(g->lc2.ensure(n * 16));
    CK(cudaMemsetAsync(g->npartial.p, 0, 8, st));
    CK(cudaMemsetAsync(g->hist.p, 0, (size_t)(D + 1) * k * 4, st));
    CK(cudaMemsetAsync(g->lc2.p, 0, n * 16, st));
    run_maxdelta(g->dcc.as<uint32_t>(), k, g->maxd.as<uint32_t>(), st);
    SqPrep sq{nullptr};
    if (g->sq) {
        RC(prepare_sq(g, k, st));
        sq.flag = g->sqflag.as<uint8_t>();
    }
    run_hyb_prep(1, n, k, DevCount{nullptr, D}, D + 1, a, b, g->sidx.as<int32_t>(),
                 g->pivot.as<int32_t>(), g->delta.as<uint32_t>(), g->dcc.as<uint32_t>(),
                 g->maxd.as<uint32_t>(), nullptr, nullptr, g->hp.as<HybPrep>(),
                 g->npartial.as<unsigned>(), sq, st);
    run_lmask(n, W, k, g->sidx.as<int32_t>(), g->pivot.as<int32_t>(), g->dcc.as<uint32_t>(),
              g->hp.as<HybPrep>(), g->Lmask.as<uint64_t>(), nullptr, st);
    g->call_kernels += 3;
    r.hist = g->hist.as<uint32_t>();
    r.D = D;
    r.Lmask = g->Lmask.as<uint64_t>();
    r.lc2 = g->lc2.as<uint64_t>();
    if (g->sq) {
        r.sqflag = g->sqflag.as<uint8_t>();
        r.istar = g->istar.as<int32_t>();
        r.pivot = g->pivot.as<int32_t>();
        r.hcse = g->hcse.as<uint64_t>();
        r.fdist = g->fdist.as<uint32_t>();
    }
    const int cw = g->cw;
    r.ld = cw;
    for (int base = 0; base < k; base += cw) {
        const int kc = std::min(cw, k - base);
        const size_t off = chunk_offset(g, base);
        if (!g->resident) RC(run_chunk(g, src + base, kc, cw, st, off));
        r.distF = g->distF.as<uint32_t>() + off;
        r.distR = g->directed ? g->distR.as<uint32_t>() + off : nullptr;
        for (int s = 0; s < kc; s += 32) {
            r.base = base + s;
            r.sub = s;
            r.kc = std::min(32, kc - s);
            run_reduce2(r, st);
            g->call_kernels += 1;
        }
    }
    run_tail(g->hist.as<uint32_t>(), DevCount{nullptr, D}, D + 1, k, g->TN.as<uint64_t>(),
             g->TS.as<uint64_t>(), st);
    run_hyb_prep(2, n, k, DevCount{nullptr, D}, D + 1, a, b, g->sidx.as<int32_t>(),
                 g->pivot.as<int32_t>(), g->delta.as<uint32_t>(), g->dcc.as<uint32_t>(),
                 g->maxd.as<uint32_t>(), g->TN.as<uint64_t>(), g->TS.as<uint64_t>(),
                 g->hp.as<HybPrep>(), g->npartial.as<unsigned>(), SqPrep{nullptr}, st);
    g->call_kernels += 2;
    return CC_OK;
}

int estimate_chunked(cc_graph *g, int k, const cc_opts *opts, cudaStream_t st)
{
    RC(chunked_pass1(g, k, st));
    if (!opts->want_hybrid) return CC_OK;
    return chunked_hybrid(g, k, opts->eps_num, opts->eps_den, st);
}

// Finalise into device buffers (or straight into device outputs) and copy.
// Arguments of the finalisation (host only: buffers sized, no stream work).
int prepare_finalize(cc_graph *g, int k, bool hyb, const cc_opts *opts, const cc_out *out,
                     FinalizeArgs &fa)
{
    const int64_t n = g->n;
    const bool dev_out = opts->device_outputs != 0;
    std::memset(&fa, 0, sizeof(fa));
    fa.n = n;
    fa.k = k;
    fa.hybrid = hyb;
    fa.sidx = g->sidx.as<int32_t>();
    fa.pivot = g->pivot.as<int32_t>();
    fa.delta = g->delta.as<uint32_t>();
    fa.sum2 = g->sum2.as<uint64_t>();
    fa.S_samp = g->Ssamp.as<uint64_t>();
    fa.lc2 = g->lc2.as<uint64_t>();
    fa.hp = g->hp.as<HybPrep>();
    if (dev_out) {
        for (int e = 0; e < CC_NUM_EST; ++e) {
            fa.s_hat[e] = out->s_hat[e];
            fa.clo[e] = out->closeness[e];
        }
        fa.hyb_int = out->hyb_int;
        fa.sample_sum = out->sample_sum;
        fa.pivot_out = out->pivot;
        fa.delta_out = (uint32_t *)out->delta;
    } else {
        // Host outputs come from library buffers, copied after the kernel
        // (the copy engines move them faster than the kernel's own stores
        // into pinned host memory: 1.36 against 1.94 ms per headline call).
        RC(g->shat.ensure((size_t)n * 8 * CC_NUM_EST));
        RC(g->clo.ensure((size_t)n * 8 * CC_NUM_EST));
        for (int e = 0; e < CC_NUM_EST; ++e) {
            fa.s_hat[e] = out->s_hat[e] ? g->shat.as<double>() + (size_t)e * n : nullptr;
            fa.clo[e] = out->closeness[e] ? g->clo.as<double>() + (size_t)e * n : nullptr;
        }
        if (out->hyb_int) {
            RC(g->hyb.ensure((size_t)n * 48));
            fa.hyb_int = g->hyb.as<uint64_t>();
        }
        if (out->sample_sum) {
            RC(g->ssum.ensure((size_t)n * 8));
            fa.sample_sum = g->ssum.as<uint64_t>();
        }
    }
    // Division-free shortcuts (bit-identical): exact scaling by 1/k for a
    // power-of-two k, and tables of the pivoting estimators over (c, Delta).
    if ((k & (k - 1)) == 0) fa.inv_k = 1.0 / (double)k;
    {
        const bool chunked = g->weighted || g->directed;
        const int64_t ts = std::min<int64_t>(chunked ? g->D1 + 1 : g->hist_cap, 256);
        RC(g->pt_clo1.ensure((size_t)k * 16));
        RC(g->pt_est2.ensure((size_t)k * ts * 8));
        RC(g->pt_clo2.ensure((size_t)k * ts * 8));
        // Sums of the bit-packed path are at most k * D < k * hist_cap.
        const int64_t c0 = chunked ? 0 : std::min<int64_t>((int64_t)k * g->hist_cap, 1 << 20);
        if (c0) RC(g->pt_clo0.ensure((size_t)c0 * 16));
        fa.clo1 = g->pt_clo1.as<double>();
        fa.est2t = g->pt_est2.as<double>();
        fa.clo2t = g->pt_clo2.as<double>();
        fa.tstride = ts;
        fa.clo0t = c0 ? g->pt_clo0.as<double>() : nullptr;
        fa.c0len = c0;
    }
    if (g->sq && hyb) {
        if (dev_out) {
            fa.sq_err = out->sq_err;
        } else {
            RC(g->sqe.ensure((size_t)n * 8));
            fa.sq_err = g->sqe.as<double>();
        }
        fa.hcse = g->hcse.as<uint64_t>();
        fa.fdist = g->fdist.as<uint32_t>();
        fa.dcc = g->dcc.as<uint32_t>();
        fa.istar = g->istar.as<int32_t>();
    }
    // Every buffer the finalisation reads must exist by now (the passes and
    // the hybrid's preparation size them); never launch it otherwise.
    if (!fa.sidx || !fa.pivot || !fa.delta || !fa.sum2 || !fa.S_samp ||
        (hyb && (!fa.lc2 || !fa.hp)) ||
        (fa.sq_err && (!fa.hcse || !fa.fdist || !fa.dcc || !fa.istar)))
        return CC_ERR_CUDA;
    return CC_OK;
}

// The estimator tables and the finalisation kernel (stream work only).
void enqueue_finalize(cc_graph *g, int k, const FinalizeArgs &fa, cudaStream_t st)
{
    const bool chunked = g->weighted || g->directed;
    const DevCount D = chunked ? DevCount{nullptr, g->D1} : DevCount{&g->ctl.as<Ctl>()->levels, 0};
    run_pivot_tables(g->n, k, g->Ssamp.as<uint64_t>(), D, fa.tstride, g->pt_clo1.as<double>(),
                     g->pt_est2.as<double>(), g->pt_clo2.as<double>(), fa.inv_k, fa.c0len,
                     fa.c0len ? g->pt_clo0.as<double>() : nullptr, st);
    run_finalize(fa, st);
    g->call_kernels += 2;
}

// Copies of the outputs the caller asked for (to the host, or between
// device buffers), then the stream is synchronised.
int copy_outputs(cc_graph *g, int k, bool hyb, const cc_opts *opts, cc_out *out,
                 const FinalizeArgs &fa, cudaStream_t st)
{
    const int64_t n = g->n;
    const bool dev_out = opts->device_outputs != 0;
    const cudaMemcpyKind kind = dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (!dev_out) {
        for (int e = 0; e < CC_NUM_EST; ++e) {
            if (e == CC_EST_HYBRID && !hyb) continue;
            if (out->s_hat[e])
                CK(cudaMemcpyAsync(out->s_hat[e], fa.s_hat[e], n * 8, kind, st));
            if (out->closeness[e])
                CK(cudaMemcpyAsync(out->closeness[e], fa.clo[e], n * 8, kind, st));
        }
        if (out->hyb_int && hyb)
            CK(cudaMemcpyAsync(out->hyb_int, fa.hyb_int, n * 48, kind, st));
        if (out->sample_sum)
            CK(cudaMemcpyAsync(out->sample_sum, fa.sample_sum, n * 8, kind, st));
        if (fa.sq_err) CK(cudaMemcpyAsync(out->sq_err, fa.sq_err, n * 8, kind, st));
    }
    if (out->pivot && !fa.pivot_out)
        CK(cudaMemcpyAsync(out->pivot, g->pivot.p, n * 4, kind, st));
    if (out->delta && !fa.delta_out)
        CK(cudaMemcpyAsync(out->delta, g->delta.p, n * 4, kind, st));
    if (out->S_sampled)
        CK(cudaMemcpyAsync(out->S_sampled, g->Ssamp.p, (size_t)k * 8, kind, st));
    if (out->delta_cc)
        CK(cudaMemcpyAsync(out->delta_cc, g->dcc.p, (size_t)k * k * 4, kind, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    return CC_OK;
}

int finish_outputs(cc_graph *g, int k, bool hyb, const cc_opts *opts, cc_out *out,
                   cudaStream_t st)
{
    FinalizeArgs fa;
    RC(prepare_finalize(g, k, hyb, opts, out, fa));
    enqueue_finalize(g, k, fa, st);
    return copy_outputs(g, k, hyb, opts, out, fa, st);
}

// Everything a bit-packed estimate queues between the sample upload and the
// output copies.  The finalisation's arguments are taken after the passes
// are queued, once every buffer they point to is sized.
int enqueue_bfs_estimate(cc_graph *g, int k, bool hyb, const cc_opts *opts, const cc_out *out,
                         bool band, FinalizeArgs &fa, cudaStream_t st)
{
    run_fill_i32(g->sidx.as<int32_t>(), g->n, -1, st);
    run_scatter_sidx(g->sidx.as<int32_t>(), g->sources.as<int32_t>(), k, st);
    g->call_kernels += 2;
    RC(estimate_bfs(g, k, opts, band, st));
    RC(prepare_finalize(g, k, hyb, opts, out, fa));
    enqueue_finalize(g, k, fa, st);
    return CC_OK;
}

// The arguments a captured estimate graph depends on.
std::vector<uint64_t> est_key(const cc_graph *g, int k, const cc_opts *opts, const cc_out *out,
                              bool band)
{
    std::vector<uint64_t> key = {g_alloc_gen.load(), (uint64_t)k, (uint64_t)opts->want_hybrid,
                                 opts->eps_num, opts->eps_den, (uint64_t)opts->device_outputs,
                                 (uint64_t)g->sq, (uint64_t)band, (uint64_t)g->hist_cap,
                                 (uint64_t)g->alpha, (uint64_t)g->max_ctas};
    // The finalisation writes device outputs in place (their addresses are
    // in the graph); host outputs are copied after it, from the library's
    // buffers, so only whether each is asked for matters.
    auto put = [&](const void *q) {
        key.push_back(opts->device_outputs ? (uint64_t)(uintptr_t)q : (uint64_t)(q != nullptr));
    };
    for (int e = 0; e < CC_NUM_EST; ++e) {
        put(out->s_hat[e]);
        put(out->closeness[e]);
    }
    put(out->hyb_int);
    put(out->sample_sum);
    put(out->sq_err);
    put(out->pivot);
    put(out->delta);
    return key;
}

// A bit-packed estimate: replayed from the captured graph when the
// arguments and buffers match the capture, captured when they match the
// previous call, queued directly otherwise (and whenever capture fails).
int run_bfs_estimate(cc_graph *g, int k, bool hyb, const cc_opts *opts, cc_out *out,
                     cudaStream_t st)
{
    if (g->hist_cap == 0) g->hist_cap = (int)std::min<int64_t>(g->n + 1, 4096);
    FinalizeArgs fa;
    const bool band = use_band(g, k, opts);
    std::vector<uint64_t> key = est_key(g, k, opts, out, band);
    auto &E = g->eg;
    E.replayed = 0;
    if (E.off) {
        RC(enqueue_bfs_estimate(g, k, hyb, opts, out, band, fa, st));
        return copy_outputs(g, k, hyb, opts, out, fa, st);
    }
    if (E.exec && E.key != key) {
        cudaGraphExecDestroy(E.exec);
        E.exec = nullptr;
    }
    if (!E.exec && E.failed != key && E.seen == key) {
        // Same arguments and buffers as the previous call: capture once.
        if (!E.cap) CK(cudaStreamCreateWithFlags(&E.cap, cudaStreamNonBlocking));
        const int kernels0 = g->call_kernels;
        bool ok = cudaStreamBeginCapture(E.cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) ok = enqueue_bfs_estimate(g, k, hyb, opts, out, band, fa, E.cap) == CC_OK;
        cudaGraph_t gr = nullptr;
        if (cudaStreamEndCapture(E.cap, &gr) != cudaSuccess) ok = false;
        // Buffers must not have moved during the capture (nothing is sized
        // there once the previous call ran with the same arguments).
        ok = ok && gr && est_key(g, k, opts, out, band) == key;
        if (ok && cudaGraphInstantiate(&E.exec, gr, 0) != cudaSuccess) {
            E.exec = nullptr;
            ok = false;
        }
        if (gr) cudaGraphDestroy(gr);
        cudaGetLastError();
        if (ok) {
            E.key = key;
            E.pend = g->pend;
            E.pend_W[0] = g->pend_W[0]; E.pend_W[1] = g->pend_W[1];
            E.pend_red[0] = g->pend_red[0]; E.pend_red[1] = g->pend_red[1];
            E.kernels = g->call_kernels - kernels0;
        } else {
            E.failed = key;  // not again for these arguments
        }
        g->pend = 0;
        g->call_kernels = kernels0;
    }
    E.seen = key;
    if (E.exec) {
        // Same arguments and buffers as at the capture: sizes nothing (if
        // it did, the graph's pointers are stale and the call runs direct).
        RC(prepare_finalize(g, k, hyb, opts, out, fa));
        if (g_alloc_gen.load() != key[0]) {
            cudaGraphExecDestroy(E.exec);
            E.exec = nullptr;
        }
    }
    if (E.exec) {
        CK(cudaGraphLaunch(E.exec, st));
        E.replayed = 1;
        g->pend = E.pend;
        g->pend_W[0] = E.pend_W[0]; g->pend_W[1] = E.pend_W[1];
        g->pend_red[0] = E.pend_red[0]; g->pend_red[1] = E.pend_red[1];
        g->call_kernels += E.kernels;
    } else {
        RC(enqueue_bfs_estimate(g, k, hyb, opts, out, band, fa, st));
    }
    return copy_outputs(g, k, hyb, opts, out, fa, st);
}

}  // namespace

void ccg::note_cuda_error(cudaError_t e, const char *file, int line)
{
    static const bool on = std::getenv("CC_DEBUG") != nullptr;
    if (on) std::fprintf(stderr, "cc: %s at %s:%d\n", cudaGetErrorString(e), file, line);
}

// Point `dst` (a handle with its own workspace) at the resident CSR of
// `src`, borrowing it: used by the server's slots.
int ccg::graph_borrow(cc_graph_t dst, cc_graph_t src)
{
    if (!dst || !src) return CC_ERR_ARG;
    dst->n = src->n;
    dst->arcs = src->arcs;
    dst->directed = src->directed;
    dst->weighted = src->weighted;
    auto cp = [](DevBuf &d, const DevBuf &s) { d.p = s.p; d.cap = s.cap; };
    cp(dst->fw.rp, src->fw.rp); cp(dst->fw.col, src->fw.col); cp(dst->fw.w, src->fw.w);
    cp(dst->rv.rp, src->rv.rp); cp(dst->rv.col, src->rv.col); cp(dst->rv.w, src->rv.w);
    cp(dst->lw.rp, src->lw.rp); cp(dst->lw.col, src->lw.col); cp(dst->lw.w, src->lw.w);
    cp(dst->lw_perm, src->lw_perm); cp(dst->lw_iperm, src->lw_iperm);
    dst->has_lw = src->has_lw;
    for (int d = 0; d < 2; ++d) {
        Classes &c = d ? dst->rv.cls : dst->fw.cls;
        const Classes &s = d ? src->rv.cls : src->fw.cls;
        cp(c.L, s.L); cp(c.M, s.M); cp(c.H, s.H); cp(c.Hn, s.Hn); cp(c.Hb, s.Hb);
        cp(c.T, s.T); cp(c.Tadj, s.Tadj);
        c.nL = s.nL; c.nM = s.nM; c.nH = s.nH; c.nHch = s.nHch; c.nT = s.nT;
    }
    dst->alpha = src->alpha;
    dst->band_off = src->band_off;
    dst->sssp_delta = src->sssp_delta;
    dst->reach_words = src->reach_words;
    dst->w_mean = src->w_mean;
    dst->borrowed = true;
    return CC_OK;
}

cc_graph_t ccg::graph_new_empty() { return new (std::nothrow) cc_graph(); }

size_t ccg::graph_workspace_bytes(cc_graph_t g)
{
    const DevBuf *ws[] = {&g->vis, &g->F0, &g->F1, &g->nxt, &g->Q0, &g->Q1, &g->T, &g->tflag,
                          &g->sidx, &g->sum2, &g->pivot, &g->delta, &g->lc2, &g->Lmask, &g->hp,
                          &g->dcc, &g->hist, &g->TN, &g->TS, &g->Ssamp, &g->maxd, &g->sources,
                          &g->npartial, &g->ctl, &g->shat, &g->clo, &g->hyb, &g->ssum,
                          &g->distF, &g->distR, &g->mask, &g->best, &g->dmax, &g->errflag,
                          &g->AL0, &g->AL1, &g->ACH0, &g->ACH1, &g->fstamp, &g->AT0, &g->AT1,
                     &g->ATa0, &g->ATa1, &g->band, &g->bflag, &g->gate2, &g->hc2, &g->sp_far0, &g->sp_far1, &g->sp_far2, &g->sp_nst, &g->sp_fst,
                     &g->hcse, &g->fdist, &g->sqflag, &g->istar, &g->sqe,
                     &g->ad_est, &g->ad_sq, &g->ad_best, &g->ad_bsq, &g->ad_clo, &g->ad_choice,
                     &g->pt_clo1, &g->pt_est2, &g->pt_clo2, &g->pt_clo0,
                     &g->beta, &g->nw_keys, &g->nw_tk, &g->nw_vals, &g->nw_tv, &g->nw_pre,
                     &g->nw_flags, &g->nw_tau, &g->nw_pick, &g->nw_mu, &g->nw_bsrc,
                     &g->nw_msum, &g->nw_wsum, &g->nw_S, &g->nw_hist, &g->nw_TS, &g->nw_lc,
                     &g->nw_out, &g->rc_order, &g->rc_rank, &g->rc_cnt, &g->rc_extra,
                     &g->rc_dsum, &g->rc_T, &g->rc_qstamp, &g->rc_vis, &g->rc_F, &g->rc_nxt,
                     &g->rc_lev, &g->rc_Q0, &g->rc_Q1, &g->rc_TL, &g->rc_out};
    size_t t = 0;
    for (const DevBuf *b : ws) t += b->cap;
    return t;
}

void ccg::graph_set_max_ctas(cc_graph_t g, int c) { g->max_ctas = c; }

// Estimates from the first pass resident in g's workspace (a completed
// cc_estimate on the same sample and k): the hybrid part for this eps --
// the deferred bits resolved when that first pass classified for the same
// eps, the second pass otherwise -- and the finalisation; no first pass.
int ccg::estimate_resident(cc_graph_t g, int32_t k, const cc_opts *opts, cc_out *out)
{
    if (!g || !opts || !out) return CC_ERR_ARG;
    if (opts->eps_num == 0 || opts->eps_num > opts->eps_den) return CC_ERR_ARG;
    reset_timing(g);
    cudaStream_t st = (cudaStream_t)opts->stream;
    const bool hyb = opts->want_hybrid != 0;
    g->sq = hyb && out->sq_err != nullptr;
    const bool chunked = g->weighted || g->directed;
    int rc = CC_OK;
    if (hyb) {
        if (chunked) {
            rc = chunked_hybrid(g, k, opts->eps_num, opts->eps_den, st);
        } else {
            const bool band = !g->sq && g->band_a == opts->eps_num && g->band_b == opts->eps_den;
            rc = bfs_hybrid(g, k, opts->eps_num, opts->eps_den, st, band);
        }
    }
    if (rc == CC_OK) rc = finish_outputs(g, k, hyb, opts, out, st);  // synchronises
    if (rc != CC_OK) {
        cudaStreamSynchronize(st);
        g->pend = 0;
        return rc;
    }
    return chunked ? CC_OK : settle_passes(g);
}


int ccg::graph_view(cc_graph_t g, GraphView *v)
{
    if (!g || !v) return CC_ERR_ARG;
    v->n = g->n;
    v->arcs = g->arcs;
    v->directed = g->directed;
    v->weighted = g->weighted;
    v->rp = g->fw.rp.as<int64_t>();
    v->col = g->fw.col.as<int32_t>();
    v->L = g->fw.cls.L.as<int32_t>();
    v->T = g->fw.cls.T.as<int32_t>();
    v->Tadj = g->fw.cls.Tadj.as<int4>();
    v->nT = g->fw.cls.nT;
    v->M = g->fw.cls.M.as<int32_t>();
    v->H = g->fw.cls.H.as<int32_t>();
    v->Hn = g->fw.cls.Hn.as<int32_t>();
    v->Hb = g->fw.cls.Hb.as<int64_t>();
    v->nL = g->fw.cls.nL;
    v->nM = g->fw.cls.nM;
    v->nH = g->fw.cls.nH;
    v->nHch = g->fw.cls.nHch;
    v->alpha = g->alpha;
    return CC_OK;
}

namespace {

int device_ok()
{
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n < 1) {
        cudaGetLastError();
        return CC_ERR_NO_DEVICE;
    }
    return CC_OK;
}

}  // namespace

extern "C" {

const char *cc_strerror(int code)
{
    switch (code) {
    case CC_OK: return "ok";
    case CC_ERR_ARG: return "invalid argument";
    case CC_ERR_GRAPH: return "malformed graph";
    case CC_ERR_DISCONNECTED: return "graph not (strongly) connected: closeness undefined";
    case CC_ERR_OOM: return "out of memory";
    case CC_ERR_TIMEOUT: return "bounded device wait ran out";
    case CC_ERR_CUDA: return "CUDA runtime error";
    case CC_ERR_TOO_LARGE: return "size beyond a documented limit";
    case CC_ERR_NO_DEVICE: return "no CUDA device";
    default: return "unknown error";
    }
}

void cc_opts_default(cc_opts *o, int32_t k)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->eps_num = 1;
    o->eps_den = (uint32_t)std::max(1L, std::lround(std::sqrt((double)std::max(k, 1))));
    o->want_hybrid = 1;
}

int cc_graph_from_edges(int64_t n, int64_t m, const uint32_t *src, const uint32_t *dst,
                        const uint32_t *w, int directed, int keep_component,
                        cc_graph_t *out, int32_t *old_id_out)
{
    if (!out) return CC_ERR_ARG;
    *out = nullptr;
    RC(device_ok());
    cc_graph *g = new (std::nothrow) cc_graph();
    if (!g) return CC_ERR_OOM;
    g->directed = directed != 0;
    int rc = CC_OK;
    std::vector<int32_t> old_id;
    if (!directed) {
        // Undirected: sort, merge, components and renumbering on the device.
        DeviceCSR d;
        rc = build_csr_device(n, m, src, dst, w, keep_component != 0, d);
        if (rc == CC_OK) rc = adopt_device_csr(g, d);
        if (rc == CC_OK && w) rc = build_locality(g, d.rp_host);
        if (d.rp) cudaFree(d.rp);
        if (d.col) cudaFree(d.col);
        if (d.w) cudaFree(d.w);
        old_id.swap(d.old_id);
    } else {
        // Directed: sort, merge, G and G^T and the largest strongly connected
        // component, all on the device.
        DeviceCSR F, R;
        rc = build_csr_device_directed(n, m, src, dst, w, keep_component != 0, F, R);
        if (rc == CC_OK) {
            rc = adopt_device_csr(g, F);
            if (rc == CC_OK) rc = adopt_device_reverse(g, R);
            old_id.swap(F.old_id);
        }
        for (DeviceCSR *d : {&F, &R}) {
            if (d->rp) cudaFree(d->rp);
            if (d->col) cudaFree(d->col);
            if (d->w) cudaFree(d->w);
        }
    }
    if (rc != CC_OK) {
        free_graph(g);
        delete g;
        return rc;
    }
    if (w && m > 0) {
        double sw = 0.0;
        for (int64_t e = 0; e < m; ++e) sw += (double)w[e];
        g->w_mean = sw / (double)m;
    }
    if (old_id_out) std::memcpy(old_id_out, old_id.data(), old_id.size() * 4);
    *out = g;
    return CC_OK;
}

int cc_graph_load_csr(int64_t n, const int64_t *row_ptr, const int32_t *col,
                      const uint32_t *w, int directed, int keep_component,
                      cc_graph_t *out, int32_t *old_id_out)
{
    if (!row_ptr || n < 2) return CC_ERR_ARG;
    const int64_t m = row_ptr[n];
    if (m > 0 && !col) return CC_ERR_ARG;
    std::vector<uint32_t> s((size_t)m), d((size_t)m);
    for (int64_t u = 0; u < n; ++u) {
        if (row_ptr[u + 1] < row_ptr[u]) return CC_ERR_GRAPH;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            if (col[e] < 0) return CC_ERR_GRAPH;
            s[e] = (uint32_t)u;
            d[e] = (uint32_t)col[e];
        }
    }
    return cc_graph_from_edges(n, m, s.data(), d.data(), w, directed, keep_component, out,
                               old_id_out);
}

int cc_graph_free(cc_graph_t g)
{
    if (!g) return CC_ERR_ARG;
    free_graph(g);
    delete g;
    return CC_OK;
}

int cc_graph_info(cc_graph_t g, int64_t *n, int64_t *arcs, int *directed, int *weighted)
{
    if (!g) return CC_ERR_ARG;
    if (n) *n = g->n;
    if (arcs) *arcs = g->arcs;
    if (directed) *directed = g->directed;
    if (weighted) *weighted = g->weighted;
    return CC_OK;
}

int cc_graph_copy_csr(cc_graph_t g, int reverse, int64_t *row_ptr, int32_t *col,
                      uint32_t *w)
{
    if (!g || (reverse && !g->directed)) return CC_ERR_ARG;
    const DevCSR &c = reverse ? g->rv : g->fw;
    if (row_ptr) CK(cudaMemcpy(row_ptr, c.rp.p, (g->n + 1) * 8, cudaMemcpyDeviceToHost));
    if (col) CK(cudaMemcpy(col, c.col.p, g->arcs * 4, cudaMemcpyDeviceToHost));
    if (w && g->weighted) CK(cudaMemcpy(w, c.w.p, g->arcs * 4, cudaMemcpyDeviceToHost));
    return CC_OK;
}

int cc_last_pass_stats(cc_graph_t g, int64_t *levels, int64_t *td, int64_t *bu,
                       int64_t *edges, int64_t *words)
{
    if (!g) return CC_ERR_ARG;
    if (levels) *levels = g->last.levels;
    if (td) *td = (int64_t)g->last.td_levels;
    if (bu) *bu = (int64_t)g->last.bu_levels;
    if (edges) *edges = (int64_t)g->last.edges;
    if (words) *words = (int64_t)g->last.words;
    return CC_OK;
}

int cc_last_pass_phases(cc_graph_t g, int64_t *warp_cycles)
{
    if (!g || !warp_cycles) return CC_ERR_ARG;
    for (int p = 0; p < CC_NUM_PHASES; ++p) warp_cycles[p] = (int64_t)g->last.ph_cycles[p];
    return CC_OK;
}

int cc_set_tuning(cc_graph_t g, int32_t alpha)
{
    if (!g || alpha < 0) return CC_ERR_ARG;
    g->alpha = alpha;
    return CC_OK;
}

int cc_set_param(cc_graph_t g, int32_t param, int32_t value)
{
    if (!g) return CC_ERR_ARG;
    switch (param) {
    case CC_PARAM_ALPHA:
        if (value < 0) return CC_ERR_ARG;
        g->alpha = value;
        return CC_OK;
    case CC_PARAM_HYBRID_ONE_PASS:
        if (value != 0 && value != 1) return CC_ERR_ARG;
        g->band_off = value == 0;
        return CC_OK;
    case CC_PARAM_SSSP_DELTA:
        g->sssp_delta = value;
        return CC_OK;
    case CC_PARAM_REACH_WORDS:
        if (value < 0 || value > kReachMaxW || (value & (value - 1))) return CC_ERR_ARG;
        g->reach_words = value;
        return CC_OK;
    case CC_PARAM_ESTIMATE_GRAPH:
        if (value != 0 && value != 1) return CC_ERR_ARG;
        g->eg.off = value == 0;
        return CC_OK;
    default:
        return CC_ERR_ARG;
    }
}

int cc_last_call_graph(cc_graph_t g, int32_t *replayed)
{
    if (!g || !replayed) return CC_ERR_ARG;
    *replayed = g->eg.replayed;
    return CC_OK;
}

int cc_last_pass_trace(cc_graph_t g, int32_t max_levels, int64_t *level_ns,
                       int32_t *top_down, int64_t *frontier, int64_t *frontier_arcs,
                       int64_t *words)
{
    if (!g || max_levels < 0) return CC_ERR_ARG;
    const int L = std::min<int>(g->last.levels + 1, std::min<int>(max_levels, kTraceLevels));
    for (int l = 1; l < L; ++l) {
        const unsigned long long t1 = (l + 1 < kTraceLevels + 1) ? g->last.lvl_ns[l + 1] : 0;
        if (level_ns) level_ns[l] = t1 > g->last.lvl_ns[l] ? (int64_t)(t1 - g->last.lvl_ns[l]) : 0;
        if (top_down) top_down[l] = (int32_t)g->last.lvl_td[l];
        if (frontier) frontier[l] = (int64_t)g->last.lvl_front[l];
        if (frontier_arcs) frontier_arcs[l] = (int64_t)g->last.lvl_ef[l];
        if (words) words[l] = (int64_t)g->last.lvl_words[l];
    }
    if (L > 0) {
        if (level_ns) level_ns[0] = 0;
        if (top_down) top_down[0] = 0;
        if (frontier) frontier[0] = 0;
        if (frontier_arcs) frontier_arcs[0] = 0;
        if (words) words[0] = 0;
    }
    return L;
}

int cc_last_call_timing(cc_graph_t g, int32_t *launches, double *kernel_ms,
                        double *alg_bytes, int32_t *all_kernels)
{
    if (!g) return CC_ERR_ARG;
    if (all_kernels) *all_kernels = g->call_kernels;
    if (launches) *launches = g->call_launches;
    if (kernel_ms) *kernel_ms = g->call_ms;
    if (alg_bytes) *alg_bytes = g->call_bytes;
    return CC_OK;
}

int cc_selftest_barrier_timeout(uint64_t timeout_ns)
{
    RC(device_ok());
    int err = 0;
    RC(launch_barrier_selftest(timeout_ns, &err));
    return err;
}

int cc_estimate(cc_graph_t g, const int32_t *sample, int32_t k, const cc_opts *opts,
                cc_out *out)
{
    if (!g || !opts || !out) return CC_ERR_ARG;
    if (opts->eps_num == 0 || opts->eps_num > opts->eps_den) return CC_ERR_ARG;
    if ((opts->roundtrip != 0) != g->directed) return CC_ERR_ARG;
    RC(validate_sample(g, sample, k));
    reset_timing(g);
    cudaStream_t st = (cudaStream_t)opts->stream;
    const int64_t n = g->n;
    RC(g->sidx.ensure(n * 4));
    RC(g->sum2.ensure(n * 16));
    RC(g->pivot.ensure(n * 4));
    RC(g->delta.ensure(n * 4));
    RC(g->dcc.ensure((size_t)k * k * 4));
    RC(g->Ssamp.ensure((size_t)k * 8));
    RC(g->sources.ensure((size_t)k * 4));
    RC(g->ctl.ensure(sizeof(Ctl)));
    CK(cudaMemcpyAsync(g->sources.p, sample, (size_t)k * 4, cudaMemcpyHostToDevice, st));
    const bool hyb = opts->want_hybrid != 0;
    g->sq = hyb && out->sq_err != nullptr;
    const bool chunked = g->weighted || g->directed;
    int rc = CC_OK;
    if (chunked) {
        run_fill_i32(g->sidx.as<int32_t>(), n, -1, st);
        run_scatter_sidx(g->sidx.as<int32_t>(), g->sources.as<int32_t>(), k, st);
        g->call_kernels += 2;
        rc = estimate_chunked(g, k, opts, st);
        if (rc == CC_OK) rc = finish_outputs(g, k, hyb, opts, out, st);  // synchronises
    } else {
        rc = run_bfs_estimate(g, k, hyb, opts, out, st);  // synchronises
    }
    if (rc != CC_OK) {
        cudaStreamSynchronize(st);
        g->pend = 0;
        return rc;
    }
    if (chunked) return CC_OK;
    // The bit-packed passes were queued without waiting: account them and
    // check the first pass now.
    rc = settle_passes(g);
    const int c1 = check_pass1(g, hyb, k);
    if (rc != CC_OK) return rc;
    if (c1 == 1) return cc_estimate(g, sample, k, opts, out);  // histogram grown: again
    return c1;
}

int cc_estimate_adaptive(cc_graph_t g, const int32_t *sample, int32_t k, const cc_opts *opts,
                         int32_t n_eps, const uint32_t *eps_num, const uint32_t *eps_den,
                         double *s_hat, double *closeness, double *sq_err, int32_t *choice)
{
    static const uint32_t kNum[] = {1, 1, 1, 1, 1, 1, 99};
    static const uint32_t kDen[] = {1000, 40, 20, 10, 5, 2, 100};
    if (!g || !opts) return CC_ERR_ARG;
    if (!eps_num || !eps_den) {
        if (eps_num || eps_den) return CC_ERR_ARG;
        n_eps = 7;
        eps_num = kNum;
        eps_den = kDen;
    }
    if (n_eps < 1 || n_eps > 64) return CC_ERR_ARG;
    for (int e = 0; e < n_eps; ++e)
        if (eps_num[e] == 0 || eps_num[e] > eps_den[e]) return CC_ERR_ARG;
    if ((opts->roundtrip != 0) != g->directed) return CC_ERR_ARG;
    RC(validate_sample(g, sample, k));
    reset_timing(g);
    cudaStream_t st = (cudaStream_t)opts->stream;
    const int64_t n = g->n;
    RC(g->sidx.ensure(n * 4));
    RC(g->sum2.ensure(n * 16));
    RC(g->pivot.ensure(n * 4));
    RC(g->delta.ensure(n * 4));
    RC(g->dcc.ensure((size_t)k * k * 4));
    RC(g->Ssamp.ensure((size_t)k * 8));
    RC(g->sources.ensure((size_t)k * 4));
    RC(g->ctl.ensure(sizeof(Ctl)));
    RC(g->ad_est.ensure((size_t)n * 8));
    RC(g->ad_sq.ensure((size_t)n * 8));
    RC(g->ad_best.ensure((size_t)n * 8));
    RC(g->ad_bsq.ensure((size_t)n * 8));
    RC(g->ad_clo.ensure((size_t)n * 8));
    RC(g->ad_choice.ensure((size_t)n * 4));
    CK(cudaMemcpyAsync(g->sources.p, sample, (size_t)k * 4, cudaMemcpyHostToDevice, st));
    run_fill_i32(g->sidx.as<int32_t>(), n, -1, st);
    run_scatter_sidx(g->sidx.as<int32_t>(), g->sources.as<int32_t>(), k, st);
    g->call_kernels += 2;
    const bool chunked = g->weighted || g->directed;
    if (chunked) {
        RC(chunked_pass1(g, k, st));
    } else {
        for (;;) {
            RC(bfs_pass1(g, k, st));
            CK(cudaStreamSynchronize(st));
            RC(settle_passes(g));
            const int c1 = check_pass1(g, true, k);
            if (c1 == 1) continue;  // histogram grown: run the first pass again
            RC(c1);
            break;
        }
    }
    g->sq = true;
    for (int e = 0; e < n_eps; ++e) {
        RC(chunked ? chunked_hybrid(g, k, eps_num[e], eps_den[e], st)
                   : bfs_hybrid(g, k, eps_num[e], eps_den[e], st));
        if (!chunked) {
            CK(cudaStreamSynchronize(st));
            RC(settle_passes(g));
        }
        FinalizeArgs fa{};
        fa.n = n;
        fa.k = k;
        fa.hybrid = 1;
        fa.sidx = g->sidx.as<int32_t>();
        fa.pivot = g->pivot.as<int32_t>();
        fa.delta = g->delta.as<uint32_t>();
        fa.sum2 = g->sum2.as<uint64_t>();
        fa.S_samp = g->Ssamp.as<uint64_t>();
        fa.lc2 = g->lc2.as<uint64_t>();
        fa.hp = g->hp.as<HybPrep>();
        fa.s_hat[CC_EST_HYBRID] = g->ad_est.as<double>();
        fa.sq_err = g->ad_sq.as<double>();
        fa.hcse = g->hcse.as<uint64_t>();
        fa.fdist = g->fdist.as<uint32_t>();
        fa.dcc = g->dcc.as<uint32_t>();
        fa.istar = g->istar.as<int32_t>();
        run_finalize(fa, st);
        run_adaptive_select(n, e, g->sidx.as<int32_t>(), g->ad_est.as<double>(),
                            g->ad_sq.as<double>(), g->ad_best.as<double>(),
                            g->ad_bsq.as<double>(), g->ad_choice.as<int32_t>(), st);
        g->call_kernels += 2;
    }
    g->sq = false;
    run_closeness(n, g->ad_best.as<double>(), g->ad_clo.as<double>(), st);
    g->call_kernels += 1;
    const cudaMemcpyKind kind =
        opts->device_outputs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (s_hat) CK(cudaMemcpyAsync(s_hat, g->ad_best.p, n * 8, kind, st));
    if (closeness) CK(cudaMemcpyAsync(closeness, g->ad_clo.p, n * 8, kind, st));
    if (sq_err) CK(cudaMemcpyAsync(sq_err, g->ad_bsq.p, n * 8, kind, st));
    if (choice) CK(cudaMemcpyAsync(choice, g->ad_choice.p, n * 4, kind, st));
    CK(cudaStreamSynchronize(st));
    return CC_OK;
}

int cc_graph_set_node_weights(cc_graph_t g, const uint32_t *beta)
{
    if (!g) return CC_ERR_ARG;
    g->has_beta = false;
    g->beta_total = 0;
    if (!beta) {
        g->beta.release();
        return CC_OK;
    }
    RC(device_ok());
    const int64_t n = g->n;
    RC(g->beta.ensure((size_t)n * 4));
    RC(g->nw_msum.ensure(16));
    CK(cudaMemcpy(g->beta.p, beta, (size_t)n * 4, cudaMemcpyHostToDevice));
    uint64_t B = 0;
    RC(nw_total(g->beta.as<uint32_t>(), n, g->nw_msum.as<uint64_t>(), &B, 0));
    if (B >= (1ull << 40)) return CC_ERR_TOO_LARGE;
    g->beta_total = B;
    g->has_beta = true;
    return CC_OK;
}

namespace {

int ensure_sampler_scratch(cc_graph *g)
{
    const size_t n = (size_t)g->n;
    RC(g->nw_keys.ensure(n * 8));
    RC(g->nw_tk.ensure(n * 8));
    RC(g->nw_vals.ensure(n * 4));
    RC(g->nw_tv.ensure(n * 4));
    RC(g->nw_pre.ensure(n * 8));
    RC(g->nw_flags.ensure(n * 8));
    RC(g->nw_tau.ensure(32));
    return CC_OK;
}

}  // namespace

int cc_sample_varopt(cc_graph_t g, int32_t k, uint64_t seed, int32_t *sample_out,
                     uint64_t *tau_out)
{
    if (!g || !sample_out || !tau_out || k < 1 || k > g->n || !g->has_beta) return CC_ERR_ARG;
    RC(device_ok());
    cudaStream_t st = 0;
    const int64_t n = g->n;
    RC(ensure_sampler_scratch(g));
    RC(g->nw_pick.ensure((size_t)k * 4));
    uint64_t *tau4 = g->nw_tau.as<uint64_t>();
    RC(nw_threshold(g->beta.as<uint32_t>(), n, k, g->nw_keys.as<uint64_t>(),
                    g->nw_vals.as<uint32_t>(), g->nw_tk.as<uint64_t>(), g->nw_tv.as<uint32_t>(),
                    g->nw_pre.as<uint64_t>(), tau4, st));
    uint64_t t4[4];
    CK(cudaMemcpy(t4, tau4, sizeof(t4), cudaMemcpyDeviceToHost));
    if (t4[2] < (uint64_t)k) return CC_ERR_ARG;  // fewer than k positive weights
    if (t4[1] == 0) return CC_ERR_CUDA;           // cannot happen (see nw_threshold)
    int64_t drawn = 0;
    RC(nw_draw(g->beta.as<uint32_t>(), n, k, seed, tau4, g->nw_keys.as<uint64_t>(),
               g->nw_vals.as<uint32_t>(), g->nw_tk.as<uint64_t>(), g->nw_tv.as<uint32_t>(),
               g->nw_pre.as<uint64_t>(), g->nw_flags.as<uint64_t>(), g->nw_pick.as<int32_t>(),
               &drawn, st));
    // The draw picks the certain nodes and exactly k - (their number) others.
    if (drawn != k) return CC_ERR_CUDA;
    CK(cudaMemcpy(sample_out, g->nw_pick.p, (size_t)k * 4, cudaMemcpyDeviceToHost));
    tau_out[0] = t4[0];
    tau_out[1] = t4[1];
    return CC_OK;
}

int cc_estimate_node_weighted(cc_graph_t g, const int32_t *sample, int32_t k,
                              const uint64_t *tau, const cc_opts *opts, cc_wout *out)
{
    if (!g || !opts || !out || !tau || !g->has_beta) return CC_ERR_ARG;
    if (tau[0] == 0 || tau[1] == 0) return CC_ERR_ARG;
    const bool hyb = opts->want_hybrid != 0;
    if (hyb && (opts->eps_num == 0 || opts->eps_num > opts->eps_den)) return CC_ERR_ARG;
    if ((opts->roundtrip != 0) != g->directed) return CC_ERR_ARG;
    RC(validate_sample(g, sample, k));
    reset_timing(g);
    cudaStream_t st = (cudaStream_t)opts->stream;
    const int64_t n = g->n;
    RC(g->sidx.ensure(n * 4));
    RC(g->sum2.ensure(n * 16));
    RC(g->pivot.ensure(n * 4));
    RC(g->delta.ensure(n * 4));
    RC(g->dcc.ensure((size_t)k * k * 4));
    RC(g->Ssamp.ensure((size_t)k * 8));
    RC(g->sources.ensure((size_t)k * 4));
    RC(g->ctl.ensure(sizeof(Ctl)));
    RC(g->nw_tau.ensure(32));
    RC(g->nw_mu.ensure((size_t)k * 8));
    RC(g->nw_bsrc.ensure((size_t)k * 4));
    RC(g->nw_msum.ensure(16));
    RC(g->nw_wsum.ensure((size_t)n * 8));
    RC(g->nw_S.ensure((size_t)k * 8));
    CK(cudaMemcpyAsync(g->sources.p, sample, (size_t)k * 4, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(g->nw_tau.p, tau, 16, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(g->nw_msum.p, 0, 16, st));
    CK(cudaMemsetAsync(g->nw_wsum.p, 0, (size_t)n * 8, st));
    CK(cudaMemsetAsync(g->nw_S.p, 0, (size_t)k * 8, st));
    run_fill_i32(g->sidx.as<int32_t>(), n, -1, st);
    run_scatter_sidx(g->sidx.as<int32_t>(), g->sources.as<int32_t>(), k, st);
    run_nw_mu(k, g->sources.as<int32_t>(), g->beta.as<uint32_t>(), g->nw_tau.as<uint64_t>(),
              g->nw_bsrc.as<uint32_t>(), g->nw_mu.as<uint64_t>(),
              g->nw_msum.as<unsigned long long>(), st);
    g->call_kernels += 3;
    NwJob j;
    std::memset(&j, 0, sizeof(j));
    j.n = n;
    j.k = k;
    j.row_of = rows_renumbered(g) ? g->lw_iperm.as<int32_t>() : nullptr;
    j.beta = g->beta.as<uint32_t>();
    j.mu = g->nw_mu.as<uint64_t>();
    j.bsrc = g->nw_bsrc.as<uint32_t>();
    j.sidx = g->sidx.as<int32_t>();
    j.wsum = g->nw_wsum.as<uint64_t>();
    j.S = g->nw_S.as<unsigned long long>();
    RC(chunked_pass1(g, k, st, &j));  // binds the distance rows it allocates
    j.distF = g->distF.as<uint32_t>();
    j.distR = g->directed ? g->distR.as<uint32_t>() : nullptr;
    uint64_t ms[2] = {0, 0};
    CK(cudaMemcpyAsync(ms, g->nw_msum.p, 16, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (ms[1]) return CC_ERR_ARG;  // a sampled node of weight 0 has probability 0
    const int64_t D = g->D1;
    // Every sum below stays in 64 bits: S_beta, the tails and the H and HC
    // parts are at most B * D, the adjusted-weight sums at most ms[0] * D.
    if ((unsigned __int128)g->beta_total * (uint64_t)D >= ((unsigned __int128)1 << 63) ||
        (unsigned __int128)ms[0] * (uint64_t)D >= ((unsigned __int128)1 << 64))
        return CC_ERR_TOO_LARGE;
    if (hyb) {
        if ((double)(D + 2) * k * 8.0 > (double)kMaxHistBytes) return CC_ERR_TOO_LARGE;
        RC(g->nw_hist.ensure((size_t)(D + 1) * k * 8));
        RC(g->nw_TS.ensure((size_t)(D + 2) * k * 8));
        RC(g->nw_lc.ensure((size_t)n * 16));
        CK(cudaMemsetAsync(g->nw_hist.p, 0, (size_t)(D + 1) * k * 8, st));
        CK(cudaMemsetAsync(g->nw_lc.p, 0, (size_t)n * 16, st));
        j.pivot = g->pivot.as<int32_t>();
        j.delta = g->delta.as<uint32_t>();
        j.dcc = g->dcc.as<uint32_t>();
        j.a = opts->eps_num;
        j.b = opts->eps_den;
        j.hist = g->nw_hist.as<unsigned long long>();
        j.lc = g->nw_lc.as<uint64_t>();
        const int cw = g->cw;
        j.ld = cw;
        const int32_t *src = g->sources.as<int32_t>();
        for (int base = 0; base < k; base += cw) {
            const int kc = std::min(cw, k - base);
            const size_t off = chunk_offset(g, base);
            if (!g->resident) RC(run_chunk(g, src + base, kc, cw, st, off));
            j.distF = g->distF.as<uint32_t>() + off;
            j.distR = g->directed ? g->distR.as<uint32_t>() + off : nullptr;
            for (int s = 0; s < kc; s += 32) {
                j.base = base + s;
                j.sub = s;
                j.kc = std::min(32, kc - s);
                run_nw_reduce2(j, D, st);
                g->call_kernels += 1;
            }
        }
        run_nw_tail(g->nw_hist.as<unsigned long long>(), D, k, g->nw_TS.as<uint64_t>(), st);
        g->call_kernels += 1;
    }
    const bool dev_out = opts->device_outputs != 0;
    NwFinal f;
    std::memset(&f, 0, sizeof(f));
    f.n = n;
    f.D = D;
    f.k = k;
    f.hybrid = hyb;
    f.a = opts->eps_num;
    f.b = opts->eps_den;
    f.B = g->beta_total;
    f.tau = g->nw_tau.as<uint64_t>();
    f.sidx = g->sidx.as<int32_t>();
    f.pivot = g->pivot.as<int32_t>();
    f.delta = g->delta.as<uint32_t>();
    f.beta = g->beta.as<uint32_t>();
    f.S = g->nw_S.as<unsigned long long>();
    f.wsum = g->nw_wsum.as<uint64_t>();
    f.lc = hyb ? g->nw_lc.as<uint64_t>() : nullptr;
    f.TS = hyb ? g->nw_TS.as<uint64_t>() : nullptr;
    if (dev_out) {
        for (int e = 0; e < 2; ++e) {
            f.s_hat[e] = out->s_hat[e];
            f.clo[e] = out->closeness[e];
        }
    } else {
        RC(g->nw_out.ensure((size_t)n * 8 * 4));
        double *stage = g->nw_out.as<double>();
        for (int e = 0; e < 2; ++e) {
            f.s_hat[e] = out->s_hat[e] ? stage + (size_t)(2 * e) * n : nullptr;
            f.clo[e] = out->closeness[e] ? stage + (size_t)(2 * e + 1) * n : nullptr;
        }
    }
    run_nw_finalize(f, st);
    g->call_kernels += 1;
    CK(cudaGetLastError());
    const cudaMemcpyKind kind = dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (out->S_sampled)
        CK(cudaMemcpyAsync(out->S_sampled, g->nw_S.p, (size_t)k * 8, kind, st));
    if (!dev_out) {
        for (int e = 0; e < (hyb ? 2 : 1); ++e) {
            if (out->s_hat[e])
                CK(cudaMemcpyAsync(out->s_hat[e], f.s_hat[e], (size_t)n * 8, kind, st));
            if (out->closeness[e])
                CK(cudaMemcpyAsync(out->closeness[e], f.clo[e], (size_t)n * 8, kind, st));
        }
    }
    CK(cudaStreamSynchronize(st));
    return CC_OK;
}

int cc_reach_estimate(cc_graph_t g, int32_t k, uint64_t seed, int32_t inbound, void *stream,
                      double *avg_dist, double *reach, int32_t *count, uint64_t *dist_sum,
                      int64_t *T)
{
    if (!g || k < 1) return CC_ERR_ARG;
    RC(device_ok());
    reset_timing(g);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)g->n;
    // Group width: CC_PARAM_REACH_WORDS words (64 sources each) or the
    // default, at most what n needs and while the per-bit levels (64 W
    // uint32 per node) take at most a quarter of the free memory.
    int W = g->reach_words > 0 ? g->reach_words : kReachDefaultW;
    while (W > 1 && 64 * W >= 2 * (int64_t)g->n) W /= 2;
    {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            return CC_ERR_CUDA;
        }
        const double avail = (double)free_b + (double)g->rc_lev.cap;
        while (W > 1 && (double)n * 64.0 * W * 4.0 > avail / 4.0) W /= 2;
    }
    const DevCSR &sg = (g->directed && !inbound) ? g->rv : g->fw;
    RC(g->nw_keys.ensure(n * 8));
    RC(g->nw_tk.ensure(n * 8));
    RC(g->nw_vals.ensure(n * 4));
    RC(g->nw_tv.ensure(n * 4));
    RC(g->rc_order.ensure(n * 4));
    RC(g->rc_rank.ensure(n * 4));
    RC(g->rc_cnt.ensure(n * 4));
    RC(g->rc_extra.ensure(n));
    RC(g->rc_dsum.ensure(n * 8));
    RC(g->rc_T.ensure(n * 8));
    RC(g->rc_qstamp.ensure(n * 4));
    RC(g->rc_vis.ensure(n * W * 8));
    RC(g->rc_F.ensure(n * W * 8));
    RC(g->rc_nxt.ensure(n * W * 8));
    RC(g->rc_lev.ensure(n * 64 * W * 4));
    RC(g->rc_Q0.ensure(n * 4));
    RC(g->rc_Q1.ensure(n * 4));
    RC(g->rc_TL.ensure(n * 4));
    RC(g->rc_out.ensure(n * 16));
    RC(g->ctl.ensure(sizeof(Ctl)));
    CK(cudaMemsetAsync(g->rc_cnt.p, 0, n * 4, st));
    CK(cudaMemsetAsync(g->rc_extra.p, 0, n, st));
    CK(cudaMemsetAsync(g->rc_dsum.p, 0, n * 8, st));
    CK(cudaMemsetAsync(g->rc_T.p, 0, n * 8, st));
    CK(cudaMemsetAsync(g->rc_qstamp.p, 0, n * 4, st));
    CK(cudaMemsetAsync(g->rc_vis.p, 0, n * W * 8, st));
    CK(cudaMemsetAsync(g->rc_F.p, 0, n * W * 8, st));
    CK(cudaMemsetAsync(g->rc_nxt.p, 0, n * W * 8, st));
    if (g->weighted) CK(cudaMemsetAsync(g->rc_lev.p, 0xFF, n * 64 * W * 4, st));
    RC(reach_order(g->n, seed, g->nw_keys.as<uint64_t>(), g->nw_vals.as<uint32_t>(),
                   g->nw_tk.as<uint64_t>(), g->nw_tv.as<uint32_t>(), g->rc_order.as<int32_t>(),
                   g->rc_rank.as<int32_t>(), st));
    ReachJob j;
    std::memset(&j, 0, sizeof(j));
    j.n = g->n;
    j.k = k;
    j.W = W;
    j.rp = sg.rp.as<int64_t>();
    j.col = sg.col.as<int32_t>();
    j.w = g->weighted ? sg.w.as<uint32_t>() : nullptr;
    j.order = g->rc_order.as<int32_t>();
    j.rank = g->rc_rank.as<int32_t>();
    j.cnt = g->rc_cnt.as<int32_t>();
    j.extra = g->rc_extra.as<uint8_t>();
    j.dsum = g->rc_dsum.as<uint64_t>();
    j.T = g->rc_T.as<int64_t>();
    j.qstamp = g->rc_qstamp.as<uint32_t>();
    j.vis = g->rc_vis.as<uint64_t>();
    j.F = g->rc_F.as<uint64_t>();
    j.nxt = g->rc_nxt.as<uint64_t>();
    j.lev = g->rc_lev.as<uint32_t>();
    j.Q[0] = g->rc_Q0.as<int32_t>();
    j.Q[1] = g->rc_Q1.as<int32_t>();
    j.TL = g->rc_TL.as<int32_t>();
    j.ctl = g->ctl.as<Ctl>();
    j.timeout_ns = kTimeoutNs;
    if (!g->ev0) {
        CK(cudaEventCreate(&g->ev0));
        CK(cudaEventCreate(&g->ev1));
    }
    CK(cudaEventRecord(g->ev0, st));
    ReachStats rs{};
    RC(reach_run(j, st, &rs));
    CK(cudaEventRecord(g->ev1, st));
    CK(cudaEventSynchronize(g->ev1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    g->call_launches = 1;
    g->call_kernels += 1;
    g->call_ms = ms;
    g->last.levels = (int)rs.levels;
    double *stage = g->rc_out.as<double>();
    reach_finalize(g->n, k, g->rc_cnt.as<int32_t>(), g->rc_dsum.as<uint64_t>(),
                   g->rc_T.as<int64_t>(), stage, stage + n, st);
    g->call_kernels += 1;
    CK(cudaGetLastError());
    if (avg_dist) CK(cudaMemcpyAsync(avg_dist, stage, n * 8, cudaMemcpyDeviceToHost, st));
    if (reach) CK(cudaMemcpyAsync(reach, stage + n, n * 8, cudaMemcpyDeviceToHost, st));
    if (count) CK(cudaMemcpyAsync(count, g->rc_cnt.p, n * 4, cudaMemcpyDeviceToHost, st));
    if (dist_sum) CK(cudaMemcpyAsync(dist_sum, g->rc_dsum.p, n * 8, cudaMemcpyDeviceToHost, st));
    if (T) CK(cudaMemcpyAsync(T, g->rc_T.p, n * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return CC_OK;
}

int cc_exact(cc_graph_t g, double *closeness, uint64_t *S)
{
    if (!g) return CC_ERR_ARG;
    const int64_t n = g->n;
    cudaStream_t st = 0;
    reset_timing(g);
    std::vector<int32_t> src;
    if (g->weighted || g->directed) {
        // Every node as a source, 32 per chunk of shortest paths; S(v) is the
        // sum of the chunk distances (round trips on directed graphs).
        RC(g->sum2.ensure(n * 16));
        RC(g->ctl.ensure(sizeof(Ctl)));
        RC(g->sources.ensure((size_t)n * 4));
        const int cw = chunk_width(g, n);
        RC(g->distF.ensure((size_t)n * cw * 4));
        if (g->directed) RC(g->distR.ensure((size_t)n * cw * 4));
        RC(g->mask.ensure(n * 8));
        RC(g->Q0.ensure(n * 4));
        RC(g->Q1.ensure(n * 4));
        RC(g->errflag.ensure(4));
        RC(g->sidx.ensure(n * 4));
        src.resize(n);
        for (int64_t v = 0; v < n; ++v) src[v] = (int32_t)v;
        CK(cudaMemcpy(g->sources.p, src.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
        CK(cudaMemsetAsync(g->sum2.p, 0, n * 16, st));
        CK(cudaMemsetAsync(g->errflag.p, 0, 4, st));
        ReduceJob r;
        std::memset(&r, 0, sizeof(r));
        r.n = n;
        r.k = (int)std::min<int64_t>(n, 0x7FFFFFFF);
        r.distF = g->distF.as<uint32_t>();
        r.distR = g->directed ? g->distR.as<uint32_t>() : nullptr;
        r.row_of = rows_renumbered(g) ? g->lw_iperm.as<int32_t>() : nullptr;
        r.sidx = g->sidx.as<int32_t>();
        r.sum2 = g->sum2.as<uint64_t>();
        r.err = g->errflag.as<int>();
        r.sum_only = 1;
        r.ld = cw;
        for (int64_t base = 0; base < n; base += cw) {
            const int kc = (int)std::min<int64_t>(cw, n - base);
            RC(run_chunk(g, g->sources.as<int32_t>() + base, kc, cw, st, 0));
            for (int s = 0; s < kc; s += 32) {
                r.base = (int)base + s;
                r.sub = s;
                r.kc = std::min(32, kc - s);
                run_reduce1(r, st);
            }
        }
        int err = 0;
        CK(cudaMemcpy(&err, g->errflag.p, 4, cudaMemcpyDeviceToHost));
        if (err) return err;
    } else {
        const int kc = (int)std::min<int64_t>(n, CC_MAX_K);
        const int W = pow2_words(kc);
        RC(ensure_state(g, W));
        RC(g->sources.ensure((size_t)kc * 4));
        CK(cudaMemsetAsync(g->sum2.p, 0, n * 16, st));
        src.resize(kc);
        for (int64_t base = 0; base < n; base += kc) {
            const int kk = (int)std::min<int64_t>(kc, n - base);
            for (int i = 0; i < kk; ++i) src[i] = (int32_t)(base + i);
            CK(cudaMemcpyAsync(g->sources.p, src.data(), (size_t)kk * 4,
                               cudaMemcpyHostToDevice, st));
            BfsJob j = base_job(g, W, g->fw, g->fw);
            j.k = kk;
            j.sources = g->sources.as<int32_t>();
            j.red = RED_SUM;
            RC(run_pass(g, W, j, st));
            if (g->last.ninc_final != 0) return CC_ERR_DISCONNECTED;
        }
    }
    std::vector<uint64_t> s2((size_t)n * 2);
    CK(cudaMemcpy(s2.data(), g->sum2.p, n * 16, cudaMemcpyDeviceToHost));
    for (int64_t v = 0; v < n; ++v) {
        if (S) S[v] = s2[2 * v];
        if (closeness) closeness[v] = (double)(n - 1) / (double)s2[2 * v];
    }
    return CC_OK;
}

int cc_sampling_sums_single(cc_graph_t g, const int32_t *sample, int32_t k, uint64_t *sum,
                            uint64_t *S_sampled)
{
    if (!g || !sum) return CC_ERR_ARG;
    if (g->directed || g->weighted) return CC_ERR_ARG;
    RC(validate_sample(g, sample, k));
    const int64_t n = g->n;
    cudaStream_t st = 0;
    reset_timing(g);
    RC(ensure_state(g, 1));
    RC(g->sources.ensure((size_t)k * 4));
    RC(g->hist.ensure((size_t)(n + 1) * 4));
    RC(g->Ssamp.ensure((size_t)k * 8));
    CK(cudaMemcpyAsync(g->sources.p, sample, (size_t)k * 4, cudaMemcpyHostToDevice, st));
    run_fill_i32(g->sidx.as<int32_t>(), n, -1, st);  // every node counted in hist
    CK(cudaMemsetAsync(g->sum2.p, 0, n * 16, st));
    std::vector<uint64_t> Sh(k, 0);
    std::vector<uint32_t> hist;
    for (int i = 0; i < k; ++i) {
        BfsJob j = base_job(g, 1, g->fw, g->fw);
        j.k = 1;
        j.sources = g->sources.as<int32_t>() + i;
        j.red = RED_SUM | (S_sampled ? RED_HIST : 0u);
        j.hist = g->hist.as<uint32_t>();
        j.hist_cap = (int)(n + 1);
        if (S_sampled) CK(cudaMemsetAsync(g->hist.p, 0, (size_t)(n + 1) * 4, st));
        RC(run_pass(g, 1, j, st));
        if (g->last.ninc_final != 0) return CC_ERR_DISCONNECTED;
        if (S_sampled) {
            const int D = g->last.levels;
            hist.resize(D + 1);
            CK(cudaMemcpy(hist.data(), g->hist.p, (size_t)(D + 1) * 4, cudaMemcpyDeviceToHost));
            uint64_t s = 0;
            for (int l = 1; l <= D; ++l) s += (uint64_t)l * hist[l];
            Sh[i] = s;
        }
    }
    std::vector<uint64_t> s2((size_t)n * 2);
    CK(cudaMemcpy(s2.data(), g->sum2.p, n * 16, cudaMemcpyDeviceToHost));
    for (int64_t v = 0; v < n; ++v) sum[v] = s2[2 * v];
    if (S_sampled) std::memcpy(S_sampled, Sh.data(), (size_t)k * 8);
    return CC_OK;
}

}  // extern "C"
