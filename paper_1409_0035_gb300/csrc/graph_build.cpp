// Graph to CSR on the host: symmetrise (undirected), drop self-loops, merge
// parallel arcs keeping the smallest length, keep the largest (strongly)
// connected component and renumber it 0..n'-1 in increasing original id,
// adjacency lists sorted by neighbour.  The component is what closeness is
// defined on (section 1: classic closeness needs every node reachable; for
// directed graphs round-trip closeness needs strong connectivity, section
// 6.1).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <utility>

#include "cc_internal.h"

namespace ccg {

namespace {

struct Arc {
    uint32_t v;
    uint32_t w;
};

// Counting sort of arcs by tail into a CSR, rows sorted by (head, length)
// and de-duplicated keeping the smallest length.
void make_csr(int64_t n, const std::vector<uint32_t> &tail,
              const std::vector<uint32_t> &head, const std::vector<uint32_t> *len,
              std::vector<int64_t> &rp, std::vector<int32_t> &col,
              std::vector<uint32_t> *wout)
{
    const size_t a = tail.size();
    std::vector<int64_t> cnt(n + 1, 0);
    for (size_t e = 0; e < a; ++e) cnt[tail[e] + 1]++;
    for (int64_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    std::vector<Arc> arcs(a);
    {
        std::vector<int64_t> cur(cnt.begin(), cnt.end() - 1);
        for (size_t e = 0; e < a; ++e)
            arcs[cur[tail[e]]++] = Arc{head[e], len ? (*len)[e] : 1u};
    }
    rp.assign(n + 1, 0);
    col.clear();
    col.reserve(a);
    if (wout) { wout->clear(); wout->reserve(a); }
    for (int64_t v = 0; v < n; ++v) {
        Arc *b = arcs.data() + cnt[v], *e = arcs.data() + cnt[v + 1];
        std::sort(b, e, [](const Arc &x, const Arc &y) {
            return x.v < y.v || (x.v == y.v && x.w < y.w);
        });
        for (Arc *p = b; p < e; ++p) {
            if (p != b && p->v == (p - 1)->v) continue;  // keep the shortest
            col.push_back((int32_t)p->v);
            if (wout) wout->push_back(p->w);
        }
        rp[v + 1] = (int64_t)col.size();
    }
}

// Weakly connected component labels (labels are the smallest node id of
// the component) by iterative BFS.
std::vector<int32_t> weak_components(int64_t n, const std::vector<int64_t> &rp,
                                     const std::vector<int32_t> &col)
{
    std::vector<int32_t> lab(n, -1), queue(n);
    for (int64_t s = 0; s < n; ++s) {
        if (lab[s] >= 0) continue;
        int64_t h = 0, t = 0;
        lab[s] = (int32_t)s;
        queue[t++] = (int32_t)s;
        while (h < t) {
            const int32_t u = queue[h++];
            for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
                const int32_t v = col[e];
                if (lab[v] < 0) { lab[v] = (int32_t)s; queue[t++] = v; }
            }
        }
    }
    return lab;
}

// Strongly connected components by an iterative Tarjan search; each label is
// the smallest node id of its component.
std::vector<int32_t> strong_components(int64_t n, const std::vector<int64_t> &rp,
                                       const std::vector<int32_t> &col)
{
    std::vector<int32_t> index(n, -1), low(n, 0), comp(n, -1), stack;
    std::vector<char> on(n, 0);
    std::vector<std::pair<int32_t, int64_t>> call;  // (node, next arc)
    int32_t counter = 0;
    stack.reserve(1024);
    for (int64_t s = 0; s < n; ++s) {
        if (index[s] >= 0) continue;
        call.push_back({(int32_t)s, rp[s]});
        index[s] = low[s] = counter++;
        stack.push_back((int32_t)s);
        on[s] = 1;
        while (!call.empty()) {
            const int32_t u = call.back().first;
            int64_t &e = call.back().second;
            if (e < rp[u + 1]) {
                const int32_t v = col[e++];
                if (index[v] < 0) {
                    index[v] = low[v] = counter++;
                    stack.push_back(v);
                    on[v] = 1;
                    call.push_back({v, rp[v]});
                } else if (on[v]) {
                    low[u] = std::min(low[u], index[v]);
                }
                continue;
            }
            if (low[u] == index[u]) {
                int32_t mn = u;
                size_t pos = stack.size();
                do { --pos; mn = std::min(mn, stack[pos]); } while (stack[pos] != u);
                for (size_t i = pos; i < stack.size(); ++i) {
                    comp[stack[i]] = mn;
                    on[stack[i]] = 0;
                }
                stack.resize(pos);
            }
            call.pop_back();
            if (!call.empty()) {
                const int32_t p = call.back().first;
                low[p] = std::min(low[p], low[u]);
            }
        }
    }
    return comp;
}

}  // namespace

int build_host_csr(int64_t n, int64_t m, const uint32_t *src, const uint32_t *dst,
                   const uint32_t *w, bool directed, bool keep_component, HostCSR &out)
{
    if (n < 2 || m < 0 || (m > 0 && (!src || !dst))) return CC_ERR_ARG;
    if (n > 0x7FFFFFFFLL) return CC_ERR_TOO_LARGE;
    const int64_t arcs_max = directed ? m : 2 * m;
    if (arcs_max > 0x7FFFFFFFLL) return CC_ERR_TOO_LARGE;
    std::vector<uint32_t> tail, head, len;
    try {
        tail.reserve(arcs_max);
        head.reserve(arcs_max);
        if (w) len.reserve(arcs_max);
        for (int64_t e = 0; e < m; ++e) {
            const uint32_t u = src[e], v = dst[e];
            if ((int64_t)u >= n || (int64_t)v >= n) return CC_ERR_GRAPH;
            if (w && w[e] == 0) return CC_ERR_ARG;
            if (u == v) continue;
            tail.push_back(u); head.push_back(v);
            if (w) len.push_back(w[e]);
            if (!directed) {
                tail.push_back(v); head.push_back(u);
                if (w) len.push_back(w[e]);
            }
        }
        std::vector<int64_t> rp;
        std::vector<int32_t> col;
        std::vector<uint32_t> wl;
        make_csr(n, tail, head, w ? &len : nullptr, rp, col, w ? &wl : nullptr);
        tail.clear(); tail.shrink_to_fit();
        head.clear(); head.shrink_to_fit();
        len.clear(); len.shrink_to_fit();

        std::vector<int32_t> new_id(n);
        int64_t nk = n;
        if (keep_component) {
            std::vector<int32_t> lab = directed ? strong_components(n, rp, col)
                                                : weak_components(n, rp, col);
            std::vector<int64_t> size(n, 0);
            for (int64_t v = 0; v < n; ++v) size[lab[v]]++;
            int64_t best = -1, bl = 0;
            for (int64_t c = 0; c < n; ++c)  // labels are smallest ids: first max wins ties
                if (size[c] > best) { best = size[c]; bl = c; }
            nk = 0;
            for (int64_t v = 0; v < n; ++v) new_id[v] = lab[v] == bl ? (int32_t)nk++ : -1;
        } else {
            std::iota(new_id.begin(), new_id.end(), 0);
        }
        if (nk < 2) return CC_ERR_GRAPH;
        out.n = nk;
        out.old_id.resize(nk);
        std::vector<uint32_t> t2, h2, l2;
        for (int64_t v = 0; v < n; ++v) {
            if (new_id[v] < 0) continue;
            out.old_id[new_id[v]] = (int32_t)v;
            for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
                const int32_t x = new_id[col[e]];
                if (x < 0) continue;
                t2.push_back((uint32_t)new_id[v]);
                h2.push_back((uint32_t)x);
                if (w) l2.push_back(wl[e]);
            }
        }
        make_csr(nk, t2, h2, w ? &l2 : nullptr, out.rp, out.col, w ? &out.w : nullptr);
        out.has_rev = directed;
        if (directed)
            make_csr(nk, h2, t2, w ? &l2 : nullptr, out.rrp, out.rcol, w ? &out.rw : nullptr);
    } catch (const std::bad_alloc &) {
        return CC_ERR_OOM;
    }
    return CC_OK;
}

}  // namespace ccg
