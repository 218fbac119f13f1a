// Serving all-nodes closeness estimates over a pool of resident graphs.
//
// A request names a graph of the pool, an estimator (sampling, pivoting,
// pivoting upper bound or hybrid -- section 2), k and a sample seed; its
// answer is every node's estimate.  The server keeps the graphs resident
// and runs requests with continuous batching: S slots, each a worker thread
// with its own CUDA stream, whose cooperative launches are capped at 1/S
// of the CTAs the GPU can hold of its least-resident kernel variant, so
// that the grids of all slots fit on the device together and run
// concurrently.  The sampled state of a request -- the workspace holding
// its first traversal pass (sums, pivots, Delta, distances between sampled
// nodes, histograms, and for the hybrid the classification on arrival) --
// stays resident after it, keyed by (graph, k, seed): a later request for
// the same sample, with any estimator or eps, runs only its own part (the
// finalisation, the hybrid's resolution or its second pass).  A waiting
// request is admitted, first come first served, as soon as a slot is free
// and its HBM footprint fits in what the running requests leave of the
// budget; idle resident states are evicted, least recently used first, to
// make room.  Arrival, start and finish times give each request's latency.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cc_internal.h"

using namespace ccg;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    int64_t id = 0;
    int graph = 0, est = 0, k = 0;
    uint64_t seed = 0;
    uint32_t a = 1, b = 1;
    size_t footprint = 0;
    Clock::time_point arrive, start, done;
    int status = 1;  // 1: waiting or running
    std::vector<double> s_hat, clo;
    std::vector<int32_t> pivot;
    std::vector<uint32_t> delta;
    std::vector<uint64_t> sum;
};

// Resident sampled state: a workspace handle (borrowing the graph's CSR)
// holding the first pass of (graph, k, seed).
struct State {
    int graph = 0, k = 0;
    uint64_t seed = 0;
    cc_graph_t ws = nullptr;
    std::vector<int32_t> sample;
    size_t bytes = 0;  // workspace held while idle
    bool busy = false;
    uint64_t tick = 0;
};

struct Slot {
    cudaStream_t st = nullptr;
    void *cand = nullptr;
    unsigned *cnt = nullptr;
    int32_t *dout = nullptr;
    std::thread th;
};

// Device bytes a request needs beyond the resident graph (workspace of one
// estimate: traversal words, per-node statistics, outputs, per-source
// tables).
size_t footprint(int64_t n, int k, bool directed_or_weighted, bool hybrid)
{
    int W = 1;
    while (W * 64 < k) W <<= 1;
    size_t per_node = (size_t)W * 8 * 5 + 4 * 10 + 16 * 2 + 8 * 2 + 32 + 48 + 64;
    if (hybrid) per_node += (size_t)64 * W + 1 + 16;  // band rows, flags, HC sums
    size_t b = (size_t)n * per_node + (size_t)k * k * 4 + (size_t)4096 * k * 20;
    if (directed_or_weighted) b += (size_t)n * 32 * 4 * 2 + (size_t)n * 16;
    return b;
}

}  // namespace

struct cc_server {
    std::vector<cc_graph_t> graphs;
    std::vector<int64_t> n;
    std::vector<Slot> slots;
    std::vector<std::unique_ptr<State>> states;
    size_t budget = 0, in_use = 0, resident = 0;
    uint64_t tick = 0;
    int64_t hits = 0, misses = 0;
    int slot_ctas = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> pending;
    std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
    std::vector<double> lat_ms;
    int64_t next_id = 1;
    int running = 0, peak_running = 0;
    bool stop = false;

    void worker(int s);
    State *find_idle(const Request *r);
    void evict_for(size_t need);
};

// An idle resident state of r's sample (caller holds mu).
State *cc_server::find_idle(const Request *r)
{
    for (auto &p : states)
        if (!p->busy && p->graph == r->graph && p->k == r->k && p->seed == r->seed)
            return p.get();
    return nullptr;
}

// Evict idle states, least recently used first, until `need` more bytes fit
// the budget (caller holds mu).
void cc_server::evict_for(size_t need)
{
    while (in_use + resident + need > budget) {
        size_t at = states.size();
        for (size_t i = 0; i < states.size(); ++i)
            if (!states[i]->busy && (at == states.size() || states[i]->tick < states[at]->tick))
                at = i;
        if (at == states.size()) return;
        resident -= states[at]->bytes;
        cc_graph_free(states[at]->ws);
        states.erase(states.begin() + (long)at);
    }
}

void cc_server::worker(int si)
{
    Slot &S = slots[si];
    for (;;) {
        Request *r = nullptr;
        State *E = nullptr;
        bool reuse = false;
        size_t charged = 0;
        {
            std::unique_lock<std::mutex> lk(mu);
            // the front request fits when its state is resident and idle, or
            // its footprint fits beside the running requests (idle states
            // can always be evicted)
            auto admissible = [&] {
                if (pending.empty()) return false;
                const Request *f = pending.front();
                return find_idle(f) != nullptr || in_use + f->footprint <= budget;
            };
            cv.wait(lk, [&] { return stop || admissible(); });
            if (stop && pending.empty()) return;
            if (!admissible()) continue;
            r = pending.front();
            pending.pop_front();
            E = find_idle(r);
            if (E) {
                reuse = true;
                resident -= E->bytes;
            } else {
                charged = r->footprint;
                evict_for(charged);
                auto fresh = std::make_unique<State>();
                fresh->graph = r->graph;
                fresh->k = r->k;
                fresh->seed = r->seed;
                fresh->ws = graph_new_empty();
                if (fresh->ws) graph_set_max_ctas(fresh->ws, slot_ctas);
                E = fresh.get();
                states.push_back(std::move(fresh));
            }
            E->busy = true;
            in_use += charged;
            running += 1;
            peak_running = std::max(peak_running, running);
            r->start = Clock::now();
        }
        const int64_t n = this->n[r->graph];
        int rc = E->ws ? CC_OK : CC_ERR_OOM;
        if (rc == CC_OK && !reuse) {
            rc = graph_borrow(E->ws, graphs[r->graph]);
            E->sample.resize(r->k);
            if (rc == CC_OK)
                rc = choose_sample_ws(n, r->k, r->seed, E->sample.data(), S.cand, S.cnt, S.dout,
                                      S.st);
        }
        if (rc == CC_OK) {
            r->s_hat.resize(n);
            r->clo.resize(n);
            r->pivot.resize(n);
            r->delta.resize(n);
            r->sum.resize(n);
            cc_opts o;
            cc_opts_default(&o, r->k);
            o.eps_num = r->a;
            o.eps_den = r->b;
            o.want_hybrid = r->est == CC_EST_HYBRID;
            int directed = 0;
            cc_graph_info(graphs[r->graph], nullptr, nullptr, &directed, nullptr);
            o.roundtrip = directed;
            o.stream = S.st;
            cc_out out;
            std::memset(&out, 0, sizeof(out));
            out.s_hat[r->est] = r->s_hat.data();
            out.closeness[r->est] = r->clo.data();
            out.pivot = r->pivot.data();
            out.delta = r->delta.data();
            out.sample_sum = r->sum.data();
            rc = reuse ? estimate_resident(E->ws, r->k, &o, &out)
                       : cc_estimate(E->ws, E->sample.data(), r->k, &o, &out);
        }
        const size_t held = rc == CC_OK ? graph_workspace_bytes(E->ws) : 0;
        {
            std::lock_guard<std::mutex> lk(mu);
            r->done = Clock::now();
            r->status = rc;
            in_use -= charged;
            running -= 1;
            if (reuse) hits += 1; else misses += 1;
            if (rc == CC_OK) {
                E->busy = false;
                E->bytes = held;
                E->tick = ++tick;
                resident += held;
            } else {
                for (size_t i = 0; i < states.size(); ++i)
                    if (states[i].get() == E) {
                        if (E->ws) cc_graph_free(E->ws);
                        states.erase(states.begin() + (long)i);
                        break;
                    }
            }
            lat_ms.push_back(std::chrono::duration<double, std::milli>(r->done - r->arrive).count());
        }
        cv.notify_all();
    }
}

extern "C" {

int cc_server_create(int32_t ngraphs, const cc_graph_t *graphs, int32_t slots,
                     uint64_t hbm_budget_bytes, cc_server_t *out)
{
    if (!out || ngraphs < 1 || !graphs || slots < 1 || slots > 64) return CC_ERR_ARG;
    *out = nullptr;
    auto srv = std::unique_ptr<cc_server>(new (std::nothrow) cc_server());
    if (!srv) return CC_ERR_OOM;
    for (int i = 0; i < ngraphs; ++i) {
        int64_t n = 0;
        if (!graphs[i] || cc_graph_info(graphs[i], &n, nullptr, nullptr, nullptr) != CC_OK)
            return CC_ERR_ARG;
        srv->graphs.push_back(graphs[i]);
        srv->n.push_back(n);
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return CC_ERR_CUDA;
    }
    srv->budget = hbm_budget_bytes ? (size_t)hbm_budget_bytes : free_b / 2;
    // Every slot's cooperative grid must fit on the GPU together with all
    // the others: cap each at (SMs x the smallest residency of any variant)
    // divided among the slots.
    // The persistent kernels also get one common L1/shared split (a quarter
    // of the unified memory is more than four CTAs of any of them use), so
    // that CTAs of different slots' kernels can share an SM.
    msbfs_set_carveout(25);
    mssp_set_carveout(25);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = std::min(msbfs_min_blocks_per_sm(), mssp_blocks_per_sm());
    srv->slot_ctas = std::max(1, sms * per_sm / slots);
    srv->slots.resize(slots);
    for (auto &S : srv->slots) {
        if (cudaStreamCreateWithFlags(&S.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc(&S.cand, sample_candidate_bytes()) != cudaSuccess ||
            cudaMalloc(&S.cnt, 4) != cudaSuccess ||
            cudaMalloc(&S.dout, (size_t)CC_MAX_K * 4) != cudaSuccess) {
            cudaGetLastError();
            return CC_ERR_OOM;
        }
    }
    cc_server *p = srv.release();
    for (int s = 0; s < slots; ++s) p->slots[s].th = std::thread([p, s] { p->worker(s); });
    *out = p;
    return CC_OK;
}

int cc_server_submit(cc_server_t s, int32_t graph, int32_t estimator, int32_t k, uint64_t seed,
                     uint32_t eps_num, uint32_t eps_den, int64_t *request_id)
{
    if (!s || !request_id || graph < 0 || graph >= (int)s->graphs.size()) return CC_ERR_ARG;
    if (estimator < 0 || estimator >= CC_NUM_EST || k < 1 || k > CC_MAX_K ||
        k > s->n[graph])
        return CC_ERR_ARG;
    if (eps_num == 0 || eps_num > eps_den) return CC_ERR_ARG;
    auto r = std::make_unique<Request>();
    int directed = 0, weighted = 0;
    cc_graph_info(s->graphs[graph], nullptr, nullptr, &directed, &weighted);
    r->graph = graph;
    r->est = estimator;
    r->k = k;
    r->seed = seed;
    r->a = eps_num;
    r->b = eps_den;
    r->footprint = footprint(s->n[graph], k, directed || weighted, estimator == CC_EST_HYBRID);
    if (r->footprint > s->budget) return CC_ERR_TOO_LARGE;
    r->arrive = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->id = s->next_id++;
        *request_id = r->id;
        s->pending.push_back(r.get());
        s->reqs[r->id] = std::move(r);
    }
    s->cv.notify_all();
    return CC_OK;
}

int cc_server_wait(cc_server_t s, int64_t request_id, int32_t timeout_ms)
{
    if (!s) return CC_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return CC_ERR_ARG;
    Request *r = it->second.get();
    const bool ok = s->cv.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)),
                                   [&] { return r->status != 1; });
    if (!ok) return CC_ERR_TIMEOUT;
    return r->status;
}

int cc_server_result(cc_server_t s, int64_t request_id, double *s_hat, double *closeness,
                     int32_t *pivot, uint32_t *delta, uint64_t *sample_sum,
                     double *latency_ms)
{
    if (!s) return CC_ERR_ARG;
    std::unique_ptr<Request> r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(request_id);
        if (it == s->reqs.end() || it->second->status == 1) return CC_ERR_ARG;
        r = std::move(it->second);
        s->reqs.erase(it);
    }
    if (r->status != CC_OK) return r->status;
    const size_t n = r->s_hat.size();
    if (s_hat) std::memcpy(s_hat, r->s_hat.data(), n * 8);
    if (closeness) std::memcpy(closeness, r->clo.data(), n * 8);
    if (pivot) std::memcpy(pivot, r->pivot.data(), n * 4);
    if (delta) std::memcpy(delta, r->delta.data(), n * 4);
    if (sample_sum) std::memcpy(sample_sum, r->sum.data(), n * 8);
    if (latency_ms)
        *latency_ms = std::chrono::duration<double, std::milli>(r->done - r->arrive).count();
    return CC_OK;
}

int cc_server_stats(cc_server_t s, int64_t *completed, double *p50_ms, double *p99_ms,
                    double *mean_ms, int32_t *peak_running)
{
    if (!s) return CC_ERR_ARG;
    std::vector<double> l;
    int peak = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        l = s->lat_ms;
        peak = s->peak_running;
    }
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) {
        if (l.empty()) return 0.0;
        const size_t i = (size_t)std::min<double>((double)l.size() - 1,
                                                  std::ceil(q * (double)l.size()) - 1);
        return l[i];
    };
    if (completed) *completed = (int64_t)l.size();
    if (p50_ms) *p50_ms = pct(0.50);
    if (p99_ms) *p99_ms = pct(0.99);
    if (mean_ms) {
        double t = 0;
        for (double x : l) t += x;
        *mean_ms = l.empty() ? 0.0 : t / (double)l.size();
    }
    if (peak_running) *peak_running = peak;
    return CC_OK;
}

int cc_server_cache_stats(cc_server_t s, int64_t *hits, int64_t *misses, int32_t *states,
                          uint64_t *resident_bytes)
{
    if (!s) return CC_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (hits) *hits = s->hits;
    if (misses) *misses = s->misses;
    if (states) *states = (int32_t)s->states.size();
    if (resident_bytes) *resident_bytes = (uint64_t)s->resident;
    return CC_OK;
}

int cc_server_free(cc_server_t s)
{
    if (!s) return CC_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    for (auto &S : s->slots)
        if (S.th.joinable()) S.th.join();
    for (auto &p : s->states)
        if (p->ws) cc_graph_free(p->ws);
    for (auto &S : s->slots) {
        if (S.st) cudaStreamDestroy(S.st);
        cudaFree(S.cand);
        cudaFree(S.cnt);
        cudaFree(S.dout);
    }
    delete s;
    return CC_OK;
}

}  // extern "C"
