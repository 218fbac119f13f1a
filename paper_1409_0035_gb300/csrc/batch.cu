// Many graphs, one persistent launch.
//
// A batch holds graphs of uneven size, each with its own sample (k <= 512)
// and eps.  One cooperative kernel covers the whole GPU; its CTAs are split
// into teams of equal size and every team works through a list of graphs,
// running each graph's whole estimate on its own CTAs: sample index, the
// bit-packed first pass (sums, pivots, Delta, sampled-pair distances, level
// histogram), the tail tables, the hybrid thresholds, the second pass when
// some L(v) misses a sampled node, and the FP64 finalisation -- the same
// device code as the single-graph path, with team-wide bounded barriers
// (sections 2-3 of the paper, applied to every graph of the batch).
//
// The team count and the graph-to-team assignment come from a planner:
// with autotuning it times every graph once alone (whole GPU), models a
// graph's time on a team of s CTAs as levels * c + work * G / s, assigns
// graphs to P teams longest-first for P in {1, 2, ..., 64}, then times every
// plan for real and keeps the fastest.  The launch and its
// memsets are captured once in a CUDA graph and replayed on every run.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <vector>

#include "cc_internal.h"
#include "estimate_dev.cuh"
#include "msbfs_dev.cuh"

namespace ccg {
namespace {

constexpr int kBatchMaxW = 8;  // k <= 512

struct BatchJob {
    BfsJob j;  // pass-1 configuration (pass 2 derived from it)
    int W, k, want_hybrid;
    uint32_t a, b;
    uint32_t *hist;
    int hist_cap;
    uint64_t *TN, *TS, *Ssamp;
    uint32_t *maxd;
    HybPrep *hp;
    uint64_t *Lmask, *lc2;
    unsigned *npartial;
    Ctl *ctl1, *ctl2;
    double *shat, *clo;  // 4 x n each
    uint64_t *hyb;       // n x 6
    int *status;
};

struct Team {
    int first, size, job_begin, job_end;
    Ctl *bar;
};

template <int W>
__device__ void run_job(const BatchJob &B, unsigned rank, unsigned size, Ctl *bar,
                        unsigned *s_hist)
{
    const int64_t gtid = (int64_t)rank * kBlock + threadIdx.x;
    const int64_t gthreads = (int64_t)size * kBlock;
    const int64_t n = B.j.n;
    const int k = B.k;
    const uint64_t to = B.j.timeout_ns;
    int32_t *sidx = const_cast<int32_t *>(B.j.sidx);
    d_fill_i32(sidx, n, -1, gtid, gthreads);
    if (!grid_sync(bar, rank, size, to)) return;
    d_scatter_sidx(sidx, B.j.sources, k, gtid, gthreads);
    if (!grid_sync(bar, rank, size, to)) return;

    bfs_pass<W>(B.j, rank, size, bar, s_hist);
    if (!grid_sync(bar, rank, size, to)) return;
    volatile Ctl *c1 = B.ctl1;
    if (c1->ninc_final != 0 || c1->err != 0) {
        if (gtid == 0) *B.status = c1->err == 1 ? CC_ERR_TOO_LARGE
                                  : c1->err < 0 ? c1->err
                                                : CC_ERR_DISCONNECTED;
        return;
    }
    const int D = c1->levels;
    d_S_sampled(B.hist, D, k, B.j.dcc, B.Ssamp, gtid >> 5, gthreads >> 5);
    if (B.want_hybrid) {
        for (int i = (int)rank; i < k; i += (int)size)
            d_tail_source(B.hist, D, k, B.TN, B.TS, i, D + 1);
        d_maxdelta(B.j.dcc, k, B.maxd, gtid >> 5, gthreads >> 5);
        if (!grid_sync(bar, rank, size, to)) return;
        d_hyb_prep(3, n, k, D, D + 1, B.a, B.b, B.j.sidx, B.j.pivot, B.j.delta, B.j.dcc, B.maxd,
                   B.TN, B.TS, B.hp, B.npartial, SqPrep{nullptr}, gtid, gthreads);
        if (!grid_sync(bar, rank, size, to)) return;
        if (*(volatile unsigned *)B.npartial > 0) {
            d_lmask(n, W, k, B.j.sidx, B.j.pivot, B.j.dcc, B.hp, B.Lmask, gtid, gthreads);
            if (!grid_sync(bar, rank, size, to)) return;
            BfsJob j2 = B.j;
            j2.red = RED_LC;
            j2.Lmask = B.Lmask;
            j2.lc2 = B.lc2;
            j2.ctl = B.ctl2;
            bfs_pass<W>(j2, rank, size, bar, s_hist);
            if (!grid_sync(bar, rank, size, to)) return;
        }
    }
    FinalizeArgs fa{};
    fa.n = n;
    fa.k = k;
    fa.hybrid = B.want_hybrid;
    fa.sidx = B.j.sidx;
    fa.pivot = B.j.pivot;
    fa.delta = B.j.delta;
    fa.sum2 = B.j.sum2;
    fa.S_samp = B.Ssamp;
    fa.lc2 = B.lc2;
    fa.hp = B.hp;
    for (int e = 0; e < CC_NUM_EST; ++e) {
        fa.s_hat[e] = B.shat + (int64_t)e * n;
        fa.clo[e] = B.clo + (int64_t)e * n;
    }
    fa.hyb_int = B.want_hybrid ? B.hyb : nullptr;
    fa.sample_sum = nullptr;
    d_finalize(fa, gtid, gthreads);
    if (!grid_sync(bar, rank, size, to)) return;
    if (gtid == 0) *B.status = CC_OK;
}

__global__ void __launch_bounds__(kBlock, 2)
batch_kernel(const BatchJob *jobs, const Team *teams, const int *cta_team, const int *order)
{
    extern __shared__ unsigned s_hist[];  // kBatchMaxW * 64 counters
    const Team T = teams[cta_team[blockIdx.x]];
    const unsigned rank = blockIdx.x - (unsigned)T.first;
    for (int q = T.job_begin; q < T.job_end; ++q) {
        const BatchJob &B = jobs[order[q]];
        switch (B.W) {
        case 1: run_job<1>(B, rank, (unsigned)T.size, T.bar, s_hist); break;
        case 2: run_job<2>(B, rank, (unsigned)T.size, T.bar, s_hist); break;
        case 4: run_job<4>(B, rank, (unsigned)T.size, T.bar, s_hist); break;
        default: run_job<8>(B, rank, (unsigned)T.size, T.bar, s_hist); break;
        }
        if (*(volatile int *)&T.bar->err < 0) return;
    }
}

struct DBuf {
    void *p = nullptr;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p) { o.p = nullptr; }
    ~DBuf() { if (p) cudaFree(p); }
};

}  // namespace
}  // namespace ccg

using namespace ccg;

struct cc_batch {
    int ngraphs = 0;
    std::vector<cc_graph_t> graphs;
    std::vector<int> k, W;
    std::vector<int64_t> n;
    std::vector<std::vector<DBuf>> bufs;  // per graph
    std::vector<BatchJob> hjobs;
    DBuf djobs, dteams, dcta, dorder, dctl, dstatus;
    size_t ctl_bytes = 0;
    int grid = 0, teams = 0;
    std::vector<double> solo_ms;
    std::vector<int> levels;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool captured = false;
    cudaStream_t cap_stream = nullptr;
    double last_ms = 0.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
};

namespace {

#define B_CK(x)                      \
    do {                             \
        if ((x) != cudaSuccess) {    \
            cudaGetLastError();      \
            return CC_ERR_CUDA;      \
        }                            \
    } while (0)
#define B_RC(x)                      \
    do {                             \
        int r_ = (x);                \
        if (r_ != CC_OK) return r_;  \
    } while (0)

int dalloc(DBuf &b, size_t bytes)
{
    if (cudaMalloc(&b.p, bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return CC_ERR_OOM;
    }
    return CC_OK;
}

int batch_grid(int *grid)
{
    int dev = 0, sms = 0, per = 0;
    B_CK(cudaGetDevice(&dev));
    B_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    B_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_kernel, kBlock,
                                                       kBatchMaxW * 64 * sizeof(unsigned)));
    if (per < 1) return CC_ERR_CUDA;
    *grid = per * sms;
    return CC_OK;
}

// Plan: P equal teams, graphs assigned longest-first to the least loaded
// team under the model t_g(s) = levels_g * c + work_g * G / s.
double plan(const cc_batch *b, int P, std::vector<int> &team_of)
{
    const double c_level = 0.012;  // ms of fixed cost per level (barriers)
    const int G = b->grid, s = G / P;
    std::vector<double> t(b->ngraphs);
    for (int i = 0; i < b->ngraphs; ++i) {
        const double fixed = b->levels[i] * c_level;
        const double work = std::max(0.0, b->solo_ms[i] - fixed);
        t[i] = fixed + work * (double)G / s;
    }
    std::vector<int> idx(b->ngraphs);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int x, int y) { return t[x] > t[y]; });
    std::vector<double> load(P, 0.0);
    team_of.assign(b->ngraphs, 0);
    for (int i : idx) {
        const int best = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        team_of[i] = best;
        load[best] += t[i];
    }
    return *std::max_element(load.begin(), load.end());
}

int upload_plan(cc_batch *b, int P, const std::vector<int> &team_of)
{
    const int G = b->grid, s = G / P;
    std::vector<Team> teams(P);
    std::vector<int> order;
    std::vector<int> cta(G, P - 1);
    for (int t = 0; t < P; ++t) {
        teams[t].first = t * s;
        teams[t].size = (t == P - 1) ? G - t * s : s;
        teams[t].job_begin = (int)order.size();
        for (int i = 0; i < b->ngraphs; ++i)
            if (team_of[i] == t) order.push_back(i);
        teams[t].job_end = (int)order.size();
        teams[t].bar = reinterpret_cast<Ctl *>(b->dctl.p) + t;
        for (int c = teams[t].first; c < teams[t].first + teams[t].size; ++c) cta[c] = t;
    }
    if (b->dteams.p) { cudaFree(b->dteams.p); b->dteams.p = nullptr; }
    if (b->dcta.p) { cudaFree(b->dcta.p); b->dcta.p = nullptr; }
    if (b->dorder.p) { cudaFree(b->dorder.p); b->dorder.p = nullptr; }
    B_RC(dalloc(b->dteams, sizeof(Team) * P));
    B_RC(dalloc(b->dcta, sizeof(int) * G));
    B_RC(dalloc(b->dorder, sizeof(int) * std::max(1, (int)order.size())));
    B_CK(cudaMemcpy(b->dteams.p, teams.data(), sizeof(Team) * P, cudaMemcpyHostToDevice));
    B_CK(cudaMemcpy(b->dcta.p, cta.data(), sizeof(int) * G, cudaMemcpyHostToDevice));
    B_CK(cudaMemcpy(b->dorder.p, order.data(), sizeof(int) * order.size(),
                    cudaMemcpyHostToDevice));
    b->teams = P;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->captured = false;
    return CC_OK;
}

// Memsets and the launch, in stream order.
int enqueue(cc_batch *b, cudaStream_t st)
{
    B_CK(cudaMemsetAsync(b->dctl.p, 0, b->ctl_bytes, st));
    B_CK(cudaMemsetAsync(b->dstatus.p, 0xFF, sizeof(int) * b->ngraphs, st));
    for (int i = 0; i < b->ngraphs; ++i) {
        const BatchJob &J = b->hjobs[i];
        const int64_t n = b->n[i];
        const int k = b->k[i];
        B_CK(cudaMemsetAsync(J.j.sum2, 0, n * 16, st));
        B_CK(cudaMemsetAsync(J.hist, 0, (size_t)J.hist_cap * k * 4, st));
        B_CK(cudaMemsetAsync(J.j.dcc, 0, (size_t)k * k * 4, st));
        B_CK(cudaMemsetAsync(J.lc2, 0, n * 16, st));
        B_CK(cudaMemsetAsync(J.npartial, 0, 4, st));
    }
    void *args[] = {&b->djobs.p, &b->dteams.p, &b->dcta.p, &b->dorder.p};
    B_CK(cudaLaunchCooperativeKernel((const void *)batch_kernel, dim3(b->grid), dim3(kBlock),
                                     args, kBatchMaxW * 64 * sizeof(unsigned), st));
    return CC_OK;
}

int run_once(cc_batch *b, cudaStream_t st, bool use_graph)
{
    if (!b->e0) {
        B_CK(cudaEventCreate(&b->e0));
        B_CK(cudaEventCreate(&b->e1));
    }
    if (use_graph && !b->captured) {
        // Capture on a private stream; fall back to direct launches when the
        // runtime refuses to capture the cooperative launch.
        if (!b->cap_stream) B_CK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
        bool ok = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal) ==
                  cudaSuccess;
        if (ok) ok = enqueue(b, b->cap_stream) == CC_OK;
        cudaGraph_t g = nullptr;
        if (cudaStreamEndCapture(b->cap_stream, &g) != cudaSuccess) ok = false;
        if (ok && g && cudaGraphInstantiate(&b->exec, g, 0) == cudaSuccess) {
            b->graph = g;
            b->captured = true;
        } else {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
        }
    }
    B_CK(cudaEventRecord(b->e0, st));
    if (use_graph && b->captured) {
        B_CK(cudaGraphLaunch(b->exec, st));
    } else {
        B_RC(enqueue(b, st));
    }
    B_CK(cudaEventRecord(b->e1, st));
    B_CK(cudaStreamSynchronize(st));
    float ms = 0.f;
    B_CK(cudaEventElapsedTime(&ms, b->e0, b->e1));
    b->last_ms = ms;
    // any barrier error (timeout) of a team
    std::vector<Ctl> bars(b->teams);
    B_CK(cudaMemcpy(bars.data(), b->dctl.p, sizeof(Ctl) * b->teams, cudaMemcpyDeviceToHost));
    for (const Ctl &c : bars)
        if (c.err < 0) return c.err;
    return CC_OK;
}

}  // namespace

extern "C" {

int cc_batch_create(int32_t ngraphs, const cc_graph_t *graphs, const int32_t *const *samples,
                    const int32_t *ks, const uint32_t *eps_num, const uint32_t *eps_den,
                    int32_t autotune, cc_batch_t *out)
{
    if (!out || ngraphs < 1 || !graphs || !samples || !ks) return CC_ERR_ARG;
    *out = nullptr;
    cc_batch *b = new (std::nothrow) cc_batch();
    if (!b) return CC_ERR_OOM;
    std::unique_ptr<cc_batch> guard(b);
    b->ngraphs = ngraphs;
    b->graphs.assign(graphs, graphs + ngraphs);
    b->bufs.resize(ngraphs);
    b->hjobs.resize(ngraphs);
    B_RC(batch_grid(&b->grid));
    const int P_max = std::min(64, b->grid);
    b->ctl_bytes = sizeof(Ctl) * (size_t)(P_max + 2 * ngraphs);
    B_RC(dalloc(b->dctl, b->ctl_bytes));
    B_RC(dalloc(b->dstatus, sizeof(int) * ngraphs));
    Ctl *ctl_jobs = reinterpret_cast<Ctl *>(b->dctl.p) + P_max;
    for (int i = 0; i < ngraphs; ++i) {
        GraphView v;
        B_RC(graph_view(graphs[i], &v));
        const int k = ks[i];
        if (v.directed || v.weighted || k < 1 || k > kBatchMaxW * 64 || k > v.n)
            return CC_ERR_ARG;
        const uint32_t a = eps_num ? eps_num[i] : 1;
        const uint32_t bb = eps_den ? eps_den[i]
                                    : (uint32_t)std::max(1L, std::lround(std::sqrt((double)k)));
        if (a == 0 || a > bb) return CC_ERR_ARG;
        std::vector<char> seen(v.n, 0);
        for (int q = 0; q < k; ++q) {
            const int32_t c = samples[i][q];
            if (c < 0 || c >= v.n || seen[c]) return CC_ERR_ARG;
            seen[c] = 1;
        }
        int W = 1;
        while (W * 64 < k) W <<= 1;
        const int64_t n = v.n;
        const int cap = (int)std::min<int64_t>(n + 1, 8192);
        b->n.push_back(n);
        b->k.push_back(k);
        b->W.push_back(W);
        auto &bf = b->bufs[i];
        bf.resize(40);
        int q = 0;
        auto take = [&](size_t bytes) -> void * {
            if (dalloc(bf[q], bytes) != CC_OK) return nullptr;
            return bf[q++].p;
        };
        BatchJob J;
        std::memset(&J, 0, sizeof(J));
        BfsJob &j = J.j;
        j.n = n;
        j.arcs = v.arcs;
        j.rp = v.rp;
        j.col = v.col;
        j.k = k;
        j.Llist = v.L; j.Mlist = v.M; j.Hlist = v.H;
        j.nL = v.nL; j.nM = v.nM; j.nH = v.nH;
        j.Tlist = v.T; j.Tadj = v.Tadj; j.nT = v.nT;
        j.Hch_node = v.Hn; j.Hch_begin = v.Hb; j.nHch = v.nHch;
        j.tHn = v.Hn; j.tHb = v.Hb; j.ntH = v.nHch;
        j.prp = v.rp; j.pcol = v.col;
        void *p[20];
        p[0] = take(n * W * 8); p[1] = take(n * W * 8); p[2] = take(n * W * 8);
        p[3] = take(n * W * 8); p[4] = take(n * 4); p[5] = take(n * 4); p[6] = take(n * 4);
        p[7] = take(n * 4); p[8] = take(n * 4); p[9] = take(n * 4); p[10] = take(n * 4);
        p[11] = take(n * 4); p[12] = take(n * 16); p[13] = take(n * 4); p[14] = take(n * 4);
        p[15] = take((size_t)k * k * 4); p[16] = take((size_t)k * 4);
        for (int z = 0; z < 17; ++z)
            if (!p[z]) return CC_ERR_OOM;
        j.vis = (uint64_t *)p[0]; j.F0 = (uint64_t *)p[1]; j.F1 = (uint64_t *)p[2];
        j.nxt = (uint64_t *)p[3];
        j.Q0 = (int32_t *)p[4]; j.Q1 = (int32_t *)p[5]; j.T = (int32_t *)p[6];
        j.tflag = (unsigned *)p[7]; j.sidx = (int32_t *)p[8]; j.AL0 = (int32_t *)p[9];
        j.AL1 = (int32_t *)p[10]; j.fstamp = (uint32_t *)p[11]; j.sum2 = (uint64_t *)p[12];
        j.pivot = (int32_t *)p[13]; j.delta = (uint32_t *)p[14]; j.dcc = (uint32_t *)p[15];
        j.dcc_k = k;
        j.sources = (int32_t *)p[16];
        j.ACH0 = (int32_t *)take((size_t)std::max<int64_t>(1, v.nHch) * 4);
        j.ACH1 = (int32_t *)take((size_t)std::max<int64_t>(1, v.nHch) * 4);
        j.AT0 = (int32_t *)take((size_t)std::max<int64_t>(1, v.nT) * 4);
        j.AT1 = (int32_t *)take((size_t)std::max<int64_t>(1, v.nT) * 4);
        j.ATa0 = (int4 *)take((size_t)std::max<int64_t>(1, v.nT) * 16);
        j.ATa1 = (int4 *)take((size_t)std::max<int64_t>(1, v.nT) * 16);
        if (!j.ACH0 || !j.ACH1 || !j.AT0 || !j.AT1 || !j.ATa0 || !j.ATa1) return CC_ERR_OOM;
        B_CK(cudaMemcpy(p[16], samples[i], (size_t)k * 4, cudaMemcpyHostToDevice));
        j.red = RED_SUM | RED_PIVOT | RED_DCC | RED_HIST;
        j.timeout_ns = 10ull * 1000 * 1000 * 1000;
        j.alpha = v.alpha ? v.alpha : default_alpha(W, j.n, j.arcs);
        j.ctl = ctl_jobs + 2 * i;
        J.W = W;
        J.k = k;
        J.want_hybrid = 1;
        J.a = a;
        J.b = bb;
        J.hist_cap = cap;
        J.hist = (uint32_t *)take((size_t)cap * k * 4);
        J.TN = (uint64_t *)take((size_t)cap * k * 8);
        J.TS = (uint64_t *)take((size_t)cap * k * 8);
        J.Ssamp = (uint64_t *)take((size_t)k * 8);
        J.maxd = (uint32_t *)take((size_t)k * 4);
        J.hp = (HybPrep *)take((size_t)n * sizeof(HybPrep));
        J.Lmask = (uint64_t *)take((size_t)n * W * 8);
        J.lc2 = (uint64_t *)take((size_t)n * 16);
        J.npartial = (unsigned *)take(4);
        J.shat = (double *)take((size_t)n * 8 * CC_NUM_EST);
        J.clo = (double *)take((size_t)n * 8 * CC_NUM_EST);
        J.hyb = (uint64_t *)take((size_t)n * 48);
        if (!J.hist || !J.TN || !J.TS || !J.Ssamp || !J.maxd || !J.hp || !J.Lmask ||
            !J.lc2 || !J.npartial || !J.shat || !J.clo || !J.hyb)
            return CC_ERR_OOM;
        j.hist = J.hist;
        j.hist_cap = cap;
        J.ctl1 = ctl_jobs + 2 * i;
        J.ctl2 = ctl_jobs + 2 * i + 1;
        J.status = reinterpret_cast<int *>(b->dstatus.p) + i;
        b->hjobs[i] = J;
    }
    B_RC(dalloc(b->djobs, sizeof(BatchJob) * ngraphs));
    B_CK(cudaMemcpy(b->djobs.p, b->hjobs.data(), sizeof(BatchJob) * ngraphs,
                    cudaMemcpyHostToDevice));

    // Cost model inputs: each graph alone on the whole GPU (autotune), or
    // arcs * W as a proxy.
    b->solo_ms.assign(ngraphs, 0.0);
    b->levels.assign(ngraphs, 0);
    if (autotune) {
        for (int i = 0; i < ngraphs; ++i) {
            cc_opts o;
            cc_opts_default(&o, b->k[i]);
            o.eps_num = b->hjobs[i].a;
            o.eps_den = b->hjobs[i].b;
            cc_out none;
            std::memset(&none, 0, sizeof(none));
            B_RC(cc_estimate(graphs[i], samples[i], b->k[i], &o, &none));
            int32_t nl = 0;
            double ms = 0, bytes = 0;
            int32_t kern = 0;
            cc_last_call_timing(graphs[i], &nl, &ms, &bytes, &kern);
            int64_t lv = 0;
            cc_last_pass_stats(graphs[i], &lv, nullptr, nullptr, nullptr, nullptr);
            b->solo_ms[i] = ms;
            b->levels[i] = (int)lv;
        }
    } else {
        for (int i = 0; i < ngraphs; ++i) {
            GraphView v;
            graph_view(graphs[i], &v);
            b->solo_ms[i] = 1e-9 * (double)v.arcs * b->W[i];
            b->levels[i] = 8;
        }
    }
    // Model every team count; with autotuning time every plan for real (the
    // model cannot tell work-bound from latency-bound graphs, whose level
    // time does not shrink with more CTAs).
    std::vector<std::pair<double, int>> cand;
    for (int P = 1; P <= P_max; P *= 2) {
        std::vector<int> t;
        cand.push_back({plan(b, P, t), P});
    }
    std::sort(cand.begin(), cand.end());
    int bestP = cand[0].second;
    if (autotune) {
        double best = 1e300;
        for (size_t c = 0; c < cand.size(); ++c) {
            std::vector<int> t;
            plan(b, cand[c].second, t);
            B_RC(upload_plan(b, cand[c].second, t));
            double tot = 0;
            for (int rep = 0; rep < 2; ++rep) {
                B_RC(run_once(b, 0, false));
                tot += b->last_ms;
            }
            if (tot < best) { best = tot; bestP = cand[c].second; }
        }
    }
    std::vector<int> team_of;
    plan(b, bestP, team_of);
    B_RC(upload_plan(b, bestP, team_of));
    *out = guard.release();
    return CC_OK;
}

int cc_batch_run(cc_batch_t b, void *stream)
{
    if (!b) return CC_ERR_ARG;
    B_RC(run_once(b, (cudaStream_t)stream, true));
    std::vector<int> st(b->ngraphs);
    B_CK(cudaMemcpy(st.data(), b->dstatus.p, sizeof(int) * b->ngraphs, cudaMemcpyDeviceToHost));
    for (int s : st)
        if (s != CC_OK) return s < 0 ? s : CC_ERR_CUDA;
    return CC_OK;
}

int cc_batch_result(cc_batch_t b, int32_t i, const cc_out *out, int32_t device_outputs)
{
    if (!b || !out || i < 0 || i >= b->ngraphs) return CC_ERR_ARG;
    const BatchJob &J = b->hjobs[i];
    const int64_t n = b->n[i];
    const int k = b->k[i];
    const cudaMemcpyKind kind = device_outputs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int e = 0; e < CC_NUM_EST; ++e) {
        if (out->s_hat[e]) B_CK(cudaMemcpy(out->s_hat[e], J.shat + (int64_t)e * n, n * 8, kind));
        if (out->closeness[e])
            B_CK(cudaMemcpy(out->closeness[e], J.clo + (int64_t)e * n, n * 8, kind));
    }
    if (out->pivot) B_CK(cudaMemcpy(out->pivot, J.j.pivot, n * 4, kind));
    if (out->delta) B_CK(cudaMemcpy(out->delta, J.j.delta, n * 4, kind));
    if (out->hyb_int) B_CK(cudaMemcpy(out->hyb_int, J.hyb, n * 48, kind));
    if (out->S_sampled) B_CK(cudaMemcpy(out->S_sampled, J.Ssamp, (size_t)k * 8, kind));
    if (out->delta_cc) B_CK(cudaMemcpy(out->delta_cc, J.j.dcc, (size_t)k * k * 4, kind));
    if (out->sample_sum) {
        std::vector<uint64_t> s2((size_t)n * 2);
        B_CK(cudaMemcpy(s2.data(), J.j.sum2, n * 16, cudaMemcpyDeviceToHost));
        std::vector<uint64_t> s(n);
        for (int64_t v = 0; v < n; ++v) s[v] = s2[2 * v];
        B_CK(cudaMemcpy(out->sample_sum, s.data(), n * 8,
                        device_outputs ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
    }
    return CC_OK;
}

int cc_batch_info(cc_batch_t b, int32_t *teams, int32_t *grid, double *last_ms,
                  int32_t *graph_captured)
{
    if (!b) return CC_ERR_ARG;
    if (teams) *teams = b->teams;
    if (grid) *grid = b->grid;
    if (last_ms) *last_ms = b->last_ms;
    if (graph_captured) *graph_captured = b->captured;
    return CC_OK;
}

int cc_batch_free(cc_batch_t b)
{
    if (!b) return CC_ERR_ARG;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->e0) cudaEventDestroy(b->e0);
    if (b->e1) cudaEventDestroy(b->e1);
    delete b;
    return CC_OK;
}

}  // extern "C"
