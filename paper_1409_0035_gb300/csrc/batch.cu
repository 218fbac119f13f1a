// Many graphs, one persistent launch per word width.
//
// A batch holds graphs of uneven size, each with its own sample (k <= 512)
// and eps.  The graphs fall into classes by their word width W (k sources
// packed in W 64-bit words per node); each class runs as one cooperative
// kernel specialised for its W that covers the whole GPU, the classes one
// after another in the same stream (and in one captured CUDA graph).  A
// class kernel's CTAs are split into teams of equal size and every team
// works through a list of graphs, running each graph's whole estimate on
// its own CTAs: sample index, the bit-packed first pass (sums, pivots,
// Delta, sampled-pair distances, level histogram, and the hybrid's
// classification on arrival), the tail tables, the hybrid thresholds, the
// resolution of the deferred bits (or the second pass when a band offset
// overflowed), and the FP64 finalisation -- the same device code as the
// single-graph path, with team-wide bounded barriers (sections 2-3 of the
// paper, applied to every graph of the batch).
//
// The autotuner (cc_batch_create with autotune = 1) times every graph
// alone under several direction switches alpha and keeps the fastest per
// graph; per class it models the time of every team count P on a team of s
// CTAs as levels * c + work * G / s (graphs longest first onto the least
// loaded team), for two block shapes (the kernel's full residency and half
// of it per SM), then times every plan for real and keeps the fastest.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "cc_internal.h"
#include "estimate_dev.cuh"
#include "msbfs_dev.cuh"

namespace ccg {
namespace {

constexpr int kBatchMaxW = 8;  // k <= 512

struct BatchJob {
    BfsJob j;   // pass 1
    BfsJob j2;  // pass 2 (the two-pass hybrid): RED_LC over Lmask
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

    // Pass 1, then (only when the hybrid needs it and the first pass could
    // not settle every bit) pass 2, from one call site.
    for (int pass = 0; pass < 2; ++pass) {
        bfs_pass<W>(pass ? B.j2 : B.j, rank, size, bar, s_hist);
        if (!grid_sync(bar, rank, size, to)) return;
        if (pass == 1) break;
        volatile Ctl *c1 = B.ctl1;
        if (c1->ninc_final != 0 || c1->err != 0) {
            if (gtid == 0) *B.status = c1->err == 1 ? CC_ERR_TOO_LARGE
                                      : c1->err < 0 ? c1->err
                                                    : CC_ERR_DISCONNECTED;
            return;
        }
        const int D = c1->levels;
        d_S_sampled(B.hist, D, k, B.j.dcc, B.Ssamp, gtid >> 5, gthreads >> 5);
        if (!B.want_hybrid) break;
        for (int i = (int)rank; i < k; i += (int)size)
            d_tail_source(B.hist, D, k, B.TN, B.TS, i, D + 1);
        d_maxdelta(B.j.dcc, k, B.maxd, gtid >> 5, gthreads >> 5);
        if (!grid_sync(bar, rank, size, to)) return;
        d_hyb_prep(3, n, k, D, D + 1, B.a, B.b, B.j.sidx, B.j.pivot, B.j.delta, B.j.dcc, B.maxd,
                   B.TN, B.TS, B.hp, B.npartial, SqPrep{nullptr}, gtid, gthreads);
        if (!grid_sync(bar, rank, size, to)) return;
        if (*(volatile unsigned *)B.npartial == 0) break;
        if (B.j.band && !c1->band_ovf) {
            // classified on arrival: resolve the deferred bits
            d_band_resolve(n, k, 64 * W, B.j.sidx, B.j.pivot, B.j.delta, B.j.dcc, B.hp,
                           B.j.bflag, B.j.band, B.j.sum2, B.lc2, B.lc2, gtid >> 5,
                           gthreads >> 5);
            if (!grid_sync(bar, rank, size, to)) return;
            break;
        }
        d_lmask(n, W, k, B.j.sidx, B.j.pivot, B.j.dcc, B.hp, B.Lmask, gtid, gthreads);
        if (!grid_sync(bar, rank, size, to)) return;
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

// Resident CTAs per SM the register allocation must allow (as the
// single-graph traversal kernel).
#ifndef CC_BATCH_MIN_CTAS
#define CC_BATCH_MIN_CTAS 4
#endif

// One word-width class: its teams (cta_team maps a CTA to its team) work
// through their graphs (order[job_begin .. job_end) of the team).
template <int W>
__global__ void __launch_bounds__(kBlock, CC_BATCH_MIN_CTAS)
    batch_kernel(const BatchJob *jobs, const Team *teams, const int *cta_team, const int *order)
{
    extern __shared__ unsigned s_hist[];  // W * 64 counters
    const Team T = teams[cta_team[blockIdx.x]];
    const unsigned rank = blockIdx.x - (unsigned)T.first;
    for (int q = T.job_begin; q < T.job_end; ++q) {
        run_job<W>(jobs[order[q]], rank, (unsigned)T.size, T.bar, s_hist);
        if (*(volatile int *)&T.bar->err < 0) return;
    }
}

constexpr int kClasses = 4;  // W = 1, 2, 4, 8
constexpr int kClassW[kClasses] = {1, 2, 4, 8};

const void *class_kernel(int c)
{
    switch (c) {
    case 0: return (const void *)batch_kernel<1>;
    case 1: return (const void *)batch_kernel<2>;
    case 2: return (const void *)batch_kernel<4>;
    default: return (const void *)batch_kernel<8>;
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

// The graphs of one word-width class and their plan.
struct BatchClass {
    std::vector<int> graphs;  // batch indices
    int grid = 0;             // CTAs of the class launch
    int per_sm = 0;           // resident CTAs per SM it uses
    int max_per_sm = 0;       // the kernel's residency limit
    int teams = 0;
    std::vector<int> team_of;  // per graph of the class
    DBuf dteams, dcta, dorder;
};

struct cc_batch {
    int ngraphs = 0;
    std::vector<cc_graph_t> graphs;
    std::vector<int> k, W, cls, alpha, cached;
    std::vector<int64_t> n;
    std::vector<std::vector<DBuf>> bufs;  // per graph
    std::vector<BatchJob> hjobs;
    BatchClass classes[kClasses];
    DBuf djobs, dctl, dstatus;
    size_t ctl_bytes = 0;
    int P_max = 64, sms = 0;
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

#define B_CK(x)                                  \
    do {                                         \
        const cudaError_t e_ = (x);              \
        if (e_ != cudaSuccess) {                 \
            note_cuda_error(e_, __FILE__, __LINE__); \
            cudaGetLastError();                  \
            return CC_ERR_CUDA;                  \
        }                                        \
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

// Streaming multiprocessors and each class kernel's resident CTAs per SM.
// ---- autotune cache ------------------------------------------------------
//
// One JSON object per line: the key (GPU name, n, arcs, k and the counts of
// the degree classes the traversal treats apart: tiny, light, medium, heavy
// nodes) and what the autotuner measured for the graph alone (the fastest
// direction switch, its device time and level count).

std::mutex g_tune_mu;
std::string g_tune_path;

struct TuneEntry {
    std::string gpu;
    int64_t n = 0, arcs = 0, k = 0, nT = 0, nL = 0, nM = 0, nH = 0;
    int64_t alpha = 0, levels = 0;
    double ms = 0;
};

bool json_num(const char *line, const char *key, double *out)
{
    char pat[64];
    std::snprintf(pat, sizeof(pat), "\"%s\":", key);
    const char *p = std::strstr(line, pat);
    if (!p) return false;
    char *end = nullptr;
    *out = std::strtod(p + std::strlen(pat), &end);
    return end != p + std::strlen(pat);
}

bool json_str(const char *line, const char *key, std::string *out)
{
    char pat[64];
    std::snprintf(pat, sizeof(pat), "\"%s\": \"", key);
    const char *p = std::strstr(line, pat);
    if (!p) return false;
    p += std::strlen(pat);
    const char *q = std::strchr(p, '"');
    if (!q) return false;
    out->assign(p, q);
    return true;
}

std::vector<TuneEntry> tune_load(const std::string &path)
{
    std::vector<TuneEntry> v;
    FILE *f = std::fopen(path.c_str(), "r");
    if (!f) return v;
    char line[1024];
    while (std::fgets(line, sizeof(line), f)) {
        TuneEntry e;
        double x[10];
        const char *keys[] = {"n", "arcs", "k", "tiny", "light", "medium", "heavy", "alpha",
                              "levels", "ms"};
        bool ok = json_str(line, "gpu", &e.gpu);
        for (int i = 0; i < 10 && ok; ++i) ok = json_num(line, keys[i], &x[i]);
        if (!ok) continue;  // not an entry of this format
        e.n = (int64_t)x[0]; e.arcs = (int64_t)x[1]; e.k = (int64_t)x[2];
        e.nT = (int64_t)x[3]; e.nL = (int64_t)x[4]; e.nM = (int64_t)x[5]; e.nH = (int64_t)x[6];
        e.alpha = (int64_t)x[7]; e.levels = (int64_t)x[8]; e.ms = x[9];
        v.push_back(e);
    }
    std::fclose(f);
    return v;
}

void tune_append(const std::string &path, const std::vector<TuneEntry> &add)
{
    if (add.empty()) return;
    FILE *f = std::fopen(path.c_str(), "a");
    if (!f) return;
    for (const TuneEntry &e : add)
        std::fprintf(f,
                     "{\"gpu\": \"%s\", \"n\": %lld, \"arcs\": %lld, \"k\": %lld, "
                     "\"tiny\": %lld, \"light\": %lld, \"medium\": %lld, \"heavy\": %lld, "
                     "\"alpha\": %lld, \"levels\": %lld, \"ms\": %.6f}\n",
                     e.gpu.c_str(), (long long)e.n, (long long)e.arcs, (long long)e.k,
                     (long long)e.nT, (long long)e.nL, (long long)e.nM, (long long)e.nH,
                     (long long)e.alpha, (long long)e.levels, e.ms);
    std::fclose(f);
}

bool same_key(const TuneEntry &a, const TuneEntry &b)
{
    return a.gpu == b.gpu && a.n == b.n && a.arcs == b.arcs && a.k == b.k && a.nT == b.nT &&
           a.nL == b.nL && a.nM == b.nM && a.nH == b.nH;
}

int batch_residency(cc_batch *b)
{
    int dev = 0;
    B_CK(cudaGetDevice(&dev));
    B_CK(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev));
    for (int c = 0; c < kClasses; ++c) {
        int per = 0;
        B_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per, class_kernel(c), kBlock, (size_t)kClassW[c] * 64 * sizeof(unsigned)));
        if (per < 1) return CC_ERR_CUDA;
        b->classes[c].max_per_sm = per;
    }
    return CC_OK;
}

// Plan of class c: P equal teams over `grid` CTAs, its graphs assigned
// longest-first to the least loaded team under the model t_g(s) =
// levels_g * c + work_g * G / s.  Returns the modelled time.
double plan(const cc_batch *b, int c, int grid, int P, std::vector<int> &team_of)
{
    const BatchClass &K = b->classes[c];
    const double c_level = 0.012;  // ms of fixed cost per level (barriers)
    const int full = b->sms * K.max_per_sm;
    const int s = grid / P;
    const int ng = (int)K.graphs.size();
    std::vector<double> t(ng);
    for (int x = 0; x < ng; ++x) {
        const int i = K.graphs[x];
        const double fixed = b->levels[i] * c_level;
        const double work = std::max(0.0, b->solo_ms[i] - fixed);
        t[x] = fixed + work * (double)full / s;
    }
    std::vector<int> idx(ng);
    std::iota(idx.begin(), idx.end(), 0);
    std::sort(idx.begin(), idx.end(), [&](int x, int y) { return t[x] > t[y]; });
    std::vector<double> load(P, 0.0);
    team_of.assign(ng, 0);
    for (int x : idx) {
        const int best = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        team_of[x] = best;
        load[best] += t[x];
    }
    return *std::max_element(load.begin(), load.end());
}

int upload_plan(cc_batch *b, int c, int per_sm, int P, const std::vector<int> &team_of)
{
    BatchClass &K = b->classes[c];
    const int G = b->sms * per_sm, s = G / P;
    std::vector<Team> teams(P);
    std::vector<int> order;
    std::vector<int> cta(G, P - 1);
    Ctl *bars = reinterpret_cast<Ctl *>(b->dctl.p) + c * b->P_max;
    for (int t = 0; t < P; ++t) {
        teams[t].first = t * s;
        teams[t].size = (t == P - 1) ? G - t * s : s;
        teams[t].job_begin = (int)order.size();
        for (size_t x = 0; x < K.graphs.size(); ++x)
            if (team_of[x] == t) order.push_back(K.graphs[x]);
        teams[t].job_end = (int)order.size();
        teams[t].bar = bars + t;
        for (int q = teams[t].first; q < teams[t].first + teams[t].size; ++q) cta[q] = t;
    }
    for (DBuf *d : {&K.dteams, &K.dcta, &K.dorder})
        if (d->p) { cudaFree(d->p); d->p = nullptr; }
    B_RC(dalloc(K.dteams, sizeof(Team) * P));
    B_RC(dalloc(K.dcta, sizeof(int) * G));
    B_RC(dalloc(K.dorder, sizeof(int) * std::max(1, (int)order.size())));
    B_CK(cudaMemcpy(K.dteams.p, teams.data(), sizeof(Team) * P, cudaMemcpyHostToDevice));
    B_CK(cudaMemcpy(K.dcta.p, cta.data(), sizeof(int) * G, cudaMemcpyHostToDevice));
    B_CK(cudaMemcpy(K.dorder.p, order.data(), sizeof(int) * order.size(),
                    cudaMemcpyHostToDevice));
    K.teams = P;
    K.grid = G;
    K.per_sm = per_sm;
    K.team_of = team_of;
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->captured = false;
    return CC_OK;
}

// Memsets and the class launches (the classes in `mask`), in stream order.
int enqueue(cc_batch *b, cudaStream_t st, unsigned mask = 0xFu)
{
    B_CK(cudaMemsetAsync(b->dctl.p, 0, b->ctl_bytes, st));
    B_CK(cudaMemsetAsync(b->dstatus.p, 0xFF, sizeof(int) * b->ngraphs, st));
    for (int i = 0; i < b->ngraphs; ++i) {
        if (!((mask >> b->cls[i]) & 1u)) continue;
        const BatchJob &J = b->hjobs[i];
        const int64_t n = b->n[i];
        const int k = b->k[i];
        B_CK(cudaMemsetAsync(J.j.sum2, 0, n * 16, st));
        B_CK(cudaMemsetAsync(J.hist, 0, (size_t)J.hist_cap * k * 4, st));
        B_CK(cudaMemsetAsync(J.j.dcc, 0, (size_t)k * k * 4, st));
        B_CK(cudaMemsetAsync(J.lc2, 0, n * 16, st));
        B_CK(cudaMemsetAsync(J.npartial, 0, 4, st));
    }
    for (int c = 0; c < kClasses; ++c) {
        BatchClass &K = b->classes[c];
        if (K.graphs.empty() || !((mask >> c) & 1u)) continue;
        void *args[] = {&b->djobs.p, &K.dteams.p, &K.dcta.p, &K.dorder.p};
        B_CK(cudaLaunchCooperativeKernel(class_kernel(c), dim3(K.grid), dim3(kBlock), args,
                                         (size_t)kClassW[c] * 64 * sizeof(unsigned), st));
    }
    return CC_OK;
}

int run_once(cc_batch *b, cudaStream_t st, bool use_graph, unsigned mask = 0xFu)
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
        B_RC(enqueue(b, st, mask));
    }
    B_CK(cudaEventRecord(b->e1, st));
    B_CK(cudaStreamSynchronize(st));
    float ms = 0.f;
    B_CK(cudaEventElapsedTime(&ms, b->e0, b->e1));
    b->last_ms = ms;
    // any barrier error (timeout) of a team
    std::vector<Ctl> bars((size_t)kClasses * b->P_max);
    B_CK(cudaMemcpy(bars.data(), b->dctl.p, sizeof(Ctl) * bars.size(), cudaMemcpyDeviceToHost));
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
    B_RC(batch_residency(b));
    b->ctl_bytes = sizeof(Ctl) * (size_t)(kClasses * b->P_max + 2 * ngraphs);
    B_RC(dalloc(b->dctl, b->ctl_bytes));
    B_RC(dalloc(b->dstatus, sizeof(int) * ngraphs));
    Ctl *ctl_jobs = reinterpret_cast<Ctl *>(b->dctl.p) + kClasses * b->P_max;
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
        const int c = W == 1 ? 0 : W == 2 ? 1 : W == 4 ? 2 : 3;
        b->cls.push_back(c);
        b->alpha.push_back(v.alpha);
        b->classes[c].graphs.push_back(i);
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
        // Rows of the hybrid's deferred bits (64W bytes per node) and their
        // flags; without them the graph takes the two-pass hybrid.
        j.band = (uint8_t *)take((size_t)n * 64 * W);
        j.bflag = j.band ? (uint8_t *)take((size_t)n) : nullptr;
        if (!j.bflag) j.band = nullptr;
        B_CK(cudaMemcpy(p[16], samples[i], (size_t)k * 4, cudaMemcpyHostToDevice));
        j.red = RED_SUM | RED_PIVOT | RED_DCC | RED_HIST | (j.band ? RED_BAND : 0u);
        j.eps_a = a;
        j.eps_b = bb;
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
        j.lc2 = J.lc2;
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
        J.j2 = j;  // every field of pass 1 set by now
        J.j2.red = RED_LC;
        J.j2.Lmask = J.Lmask;
        J.j2.lc2 = J.lc2;
        J.j2.ctl = J.ctl2;
        b->hjobs[i] = J;
    }

    // Cost model inputs: each graph alone on the whole GPU (autotune: under
    // every direction switch of the candidate list, keeping the fastest),
    // or arcs * W as a proxy.
    b->solo_ms.assign(ngraphs, 0.0);
    b->levels.assign(ngraphs, 0);
    std::string tpath;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tpath = g_tune_path;
    }
    std::vector<TuneEntry> cache, fresh;
    std::string gpu;
    if (autotune && !tpath.empty()) {
        cudaDeviceProp prop;
        int dev = 0;
        B_CK(cudaGetDevice(&dev));
        B_CK(cudaGetDeviceProperties(&prop, dev));
        gpu = prop.name;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        cache = tune_load(tpath);
    }
    b->cached.assign(ngraphs, 0);
    if (autotune) {
        const int alphas[] = {0, 2, 4, 8, 14};
        for (int i = 0; i < ngraphs; ++i) {
            TuneEntry key;
            if (!tpath.empty()) {
                GraphView v;
                B_RC(graph_view(graphs[i], &v));
                key.gpu = gpu;
                key.n = v.n; key.arcs = v.arcs; key.k = b->k[i];
                key.nT = v.nT; key.nL = v.nL; key.nM = v.nM; key.nH = v.nH;
                const TuneEntry *hit = nullptr;
                for (const TuneEntry &e : cache)
                    if (same_key(e, key)) hit = &e;  // the last entry of a key wins
                if (hit) {
                    BfsJob &j = b->hjobs[i].j;
                    b->alpha[i] = (int)hit->alpha;
                    j.alpha = b->alpha[i];
                    b->hjobs[i].j2.alpha = b->alpha[i];
                    b->solo_ms[i] = hit->ms;
                    b->levels[i] = (int)hit->levels;
                    b->cached[i] = 1;
                    continue;
                }
            }
            cc_opts o;
            cc_opts_default(&o, b->k[i]);
            o.eps_num = b->hjobs[i].a;
            o.eps_den = b->hjobs[i].b;
            cc_out none;
            std::memset(&none, 0, sizeof(none));
            const int keep = b->alpha[i];
            B_RC(cc_estimate(graphs[i], samples[i], b->k[i], &o, &none));  // warm
            double best = 1e300;
            int best_a = 0;
            int64_t best_lv = 0;
            for (int al : alphas) {
                B_RC(cc_set_tuning(graphs[i], al));
                B_RC(cc_estimate(graphs[i], samples[i], b->k[i], &o, &none));
                int32_t nl = 0, kern = 0;
                double ms = 0, bytes = 0;
                cc_last_call_timing(graphs[i], &nl, &ms, &bytes, &kern);
                int64_t lv = 0;
                cc_last_pass_stats(graphs[i], &lv, nullptr, nullptr, nullptr, nullptr);
                if (ms < best) { best = ms; best_a = al; best_lv = lv; }
            }
            B_RC(cc_set_tuning(graphs[i], keep));
            BfsJob &j = b->hjobs[i].j;
            b->alpha[i] = best_a ? best_a : default_alpha(b->W[i], j.n, j.arcs);
            j.alpha = b->alpha[i];
            b->hjobs[i].j2.alpha = b->alpha[i];
            b->solo_ms[i] = best;
            b->levels[i] = (int)best_lv;
            if (!tpath.empty()) {
                key.alpha = b->alpha[i];
                key.levels = best_lv;
                key.ms = best;
                fresh.push_back(key);
                cache.push_back(key);  // a repeated graph of this batch hits it
            }
        }
        if (!fresh.empty()) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            tune_append(tpath, fresh);
        }
    } else {
        for (int i = 0; i < ngraphs; ++i) {
            const BfsJob &j = b->hjobs[i].j;
            b->alpha[i] = j.alpha;
            b->solo_ms[i] = 1e-9 * (double)j.arcs * b->W[i];
            b->levels[i] = 8;
        }
    }
    B_RC(dalloc(b->djobs, sizeof(BatchJob) * ngraphs));
    B_CK(cudaMemcpy(b->djobs.p, b->hjobs.data(), sizeof(BatchJob) * ngraphs,
                    cudaMemcpyHostToDevice));
    // Per class: every team count P and two block shapes (the kernel's full
    // residency per SM and half of it) by the model; with autotuning the six
    // best by the model are timed for real (the model cannot tell
    // work-bound from latency-bound graphs, whose level time does not
    // shrink with more CTAs).
    for (int c = 0; c < kClasses; ++c) {
        BatchClass &K = b->classes[c];
        if (K.graphs.empty()) continue;
        struct Cand { double t; int per, P; };
        std::vector<Cand> cand;
        std::vector<int> shapes = {K.max_per_sm};
        if (K.max_per_sm / 2 >= 1 && K.max_per_sm / 2 != K.max_per_sm)
            shapes.push_back(K.max_per_sm / 2);
        for (int per : shapes) {
            const int G = b->sms * per;
            for (int P = 1; P <= std::min(b->P_max, G); P *= 2) {
                std::vector<int> t;
                cand.push_back({plan(b, c, G, P, t), per, P});
            }
        }
        std::sort(cand.begin(), cand.end(), [](const Cand &x, const Cand &y) { return x.t < y.t; });
        Cand best = cand[0];
        if (autotune) {
            double bt = 1e300;
            for (size_t q = 0; q < cand.size() && q < 6; ++q) {
                std::vector<int> t;
                plan(b, c, b->sms * cand[q].per, cand[q].P, t);
                B_RC(upload_plan(b, c, cand[q].per, cand[q].P, t));
                double tot = 0;
                for (int rep = 0; rep < 2; ++rep) {
                    B_RC(run_once(b, 0, false, 1u << c));
                    tot += b->last_ms;
                }
                if (tot < bt) { bt = tot; best = cand[q]; }
            }
        }
        std::vector<int> team_of;
        plan(b, c, b->sms * best.per, best.P, team_of);
        B_RC(upload_plan(b, c, best.per, best.P, team_of));
    }
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
    int t = 0, g = 0;
    for (const BatchClass &K : b->classes) {
        t += K.teams;
        g = std::max(g, K.grid);
    }
    if (teams) *teams = t;
    if (grid) *grid = g;
    if (last_ms) *last_ms = b->last_ms;
    if (graph_captured) *graph_captured = b->captured;
    return CC_OK;
}

int cc_batch_tune_cache(const char *path)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_path = path ? path : "";
    return CC_OK;
}

int cc_batch_plan(cc_batch_t b, int32_t i, int32_t *words, int32_t *alpha, int32_t *team,
                  int32_t *class_teams, int32_t *class_ctas, int32_t *ctas_per_sm,
                  int32_t *from_cache)
{
    if (!b || i < 0 || i >= b->ngraphs) return CC_ERR_ARG;
    if (from_cache) *from_cache = i < (int)b->cached.size() ? b->cached[i] : 0;
    const BatchClass &K = b->classes[b->cls[i]];
    int x = 0;
    while (x < (int)K.graphs.size() && K.graphs[x] != i) ++x;
    if (words) *words = b->W[i];
    if (alpha) *alpha = b->alpha[i];
    if (team) *team = x < (int)K.team_of.size() ? K.team_of[x] : 0;
    if (class_teams) *class_teams = K.teams;
    if (class_ctas) *class_ctas = K.grid;
    if (ctas_per_sm) *ctas_per_sm = K.per_sm;
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
