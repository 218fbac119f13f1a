/*
 * cc_oracle.c -- plain, slow, obviously-correct CPU oracle for the all-nodes
 * classic closeness estimators of Cohen, Delling, Pajor and Werneck,
 * "Computing Classic Closeness Centrality, at Scale" (2014).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The GPU library
 * shares no code with it: no header, helper, table or constant.
 *
 * Everything here is computed from the definitions, not from the paper's
 * streaming machinery (Algorithm 1's List/Thresh/bin arrays):
 *   - shortest-path distances by a textbook queue BFS (unit lengths) or a
 *     binary-heap Dijkstra (uint32 arc lengths >= 1), section 3;
 *   - an explicit k x n table dist[i][v] = d(c_i, v), section 2 ("the nk
 *     computed distances");
 *   - pivot c(j) = argmin_i d(c_i, j), ties to the smallest sample index,
 *     Delta(j) = d(j, c(j)), section 2;
 *   - sampling estimator, eq. (3); pivoting estimator B(c(j)) and pivoting
 *     upper bound B(c(j)) + Delta(j), section 2;
 *   - hybrid estimator, eq. (4), evaluated set by set (H, HC, L cap C);
 *   - exact S(v) = sum_u d(v,u) and B^-1(v) = (n-1)/S(v), eq. (1).
 *
 * Readings taken where the paper is silent or loose (each also listed in the
 * design notes):
 *   - eps is the rational a/b with 0 < a <= b; "d > Delta/eps" is evaluated as
 *     d*a > Delta*b in exact integers (partition boundary: strictly greater
 *     goes to H / HC, at most goes to L; section 2 definition of L(j)).
 *   - pivot ties go to the smallest sample index i (order of `sources`).
 *   - for j in C every estimator returns the exact S(j) (section 2: "for
 *     points j in C we can compute the exact value").
 *   - the sampling estimate of S(j) for j not in C is (n-1)/k * sum_i d_ij,
 *     i.e. eq. (3) scaled from B to S.
 *   - FP64 finalisation: the integer numerator is formed in unsigned 128-bit,
 *     converted to double once and divided once.
 *
 * Return codes: 0 ok, -1 bad argument, -2 distance overflow (>= 2^32-1),
 * -3 unreachable node (graph not connected), -4 out of memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF 0xFFFFFFFFu

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* Single-source shortest paths                                              */
/* ------------------------------------------------------------------------ */

/* Textbook FIFO-queue breadth-first search from s.  dist[v] = number of arcs
 * on a shortest s-v path, ORC_INF when v is unreachable.  (Section 3 runs
 * Dijkstra from each sampled node; with unit lengths that is BFS.) */
int orc_bfs(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t s,
            uint32_t *dist)
{
    if (n <= 0 || s < 0 || s >= n) return -1;
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!queue) return -4;
    for (int64_t v = 0; v < n; ++v) dist[v] = ORC_INF;
    int64_t head = 0, tail = 0;
    dist[s] = 0;
    queue[tail++] = s;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col[e];
            if (dist[v] == ORC_INF) {
                dist[v] = dist[u] + 1;
                queue[tail++] = v;
            }
        }
    }
    free(queue);
    return 0;
}

/* Binary min-heap of (distance, node) pairs, ordered lexicographically. */
typedef struct { uint64_t d; int32_t v; } heap_item;

static int heap_less(heap_item a, heap_item b)
{
    return a.d < b.d || (a.d == b.d && a.v < b.v);
}

static void heap_push(heap_item *h, int64_t *size, heap_item x)
{
    int64_t i = (*size)++;
    h[i] = x;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!heap_less(h[i], h[p])) break;
        heap_item t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}

static heap_item heap_pop(heap_item *h, int64_t *size)
{
    heap_item top = h[0];
    h[0] = h[--(*size)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < *size && heap_less(h[l], h[m])) m = l;
        if (r < *size && heap_less(h[r], h[m])) m = r;
        if (m == i) break;
        heap_item t = h[i]; h[i] = h[m]; h[m] = t;
        i = m;
    }
    return top;
}

/* Dijkstra's algorithm with a lazy-deletion binary heap keyed by
 * (distance, node).  Arc lengths w[e] >= 1 (section 7 uses 32-bit integer arc
 * lengths).  dist[v] = ORC_INF when unreachable; returns -2 when a distance
 * reaches 2^32-1 (does not fit the uint32 result). */
int orc_dijkstra(int64_t n, const int64_t *row_ptr, const int32_t *col,
                 const uint32_t *w, int32_t s, uint32_t *dist)
{
    if (n <= 0 || s < 0 || s >= n) return -1;
    int64_t m = row_ptr[n];
    uint64_t *d = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    heap_item *h = (heap_item *)malloc((size_t)(m + 1) * sizeof(heap_item));
    char *done = (char *)calloc((size_t)n, 1);
    if (!d || !h || !done) { free(d); free(h); free(done); return -4; }
    for (int64_t v = 0; v < n; ++v) d[v] = UINT64_MAX;
    int64_t size = 0;
    d[s] = 0;
    heap_item first = {0, s};
    heap_push(h, &size, first);
    while (size > 0) {
        heap_item it = heap_pop(h, &size);
        if (done[it.v]) continue;
        done[it.v] = 1;
        for (int64_t e = row_ptr[it.v]; e < row_ptr[it.v + 1]; ++e) {
            int32_t v = col[e];
            uint64_t nd = it.d + (uint64_t)w[e];
            if (nd < d[v]) {
                d[v] = nd;
                heap_item x = {nd, v};
                heap_push(h, &size, x);
            }
        }
    }
    int rc = 0;
    for (int64_t v = 0; v < n; ++v) {
        if (d[v] == UINT64_MAX) dist[v] = ORC_INF;
        else if (d[v] >= (uint64_t)ORC_INF) { dist[v] = ORC_INF; rc = -2; }
        else dist[v] = (uint32_t)d[v];
    }
    free(d); free(h); free(done);
    return rc;
}

static int sssp(int64_t n, const int64_t *row_ptr, const int32_t *col,
                const uint32_t *w, int32_t s, uint32_t *dist)
{
    return w ? orc_dijkstra(n, row_ptr, col, w, s, dist)
             : orc_bfs(n, row_ptr, col, s, dist);
}

/* table[i*n + v] = d(sources[i], v) for i in [0,k): one SSSP per sampled
 * node (section 3, first paragraph).  Returns -3 if some node is unreachable
 * from some source. */
int orc_dist_table(int64_t n, const int64_t *row_ptr, const int32_t *col,
                   const uint32_t *w, int32_t k, const int32_t *sources,
                   uint32_t *table)
{
    if (k <= 0) return -1;
    for (int32_t i = 0; i < k; ++i) {
        int rc = sssp(n, row_ptr, col, w, sources[i], table + (size_t)i * n);
        if (rc) return rc;
        for (int64_t v = 0; v < n; ++v)
            if (table[(size_t)i * n + v] == ORC_INF) return -3;
    }
    return 0;
}

/* Round-trip table (section 6.1): rt[i][v] = d(c_i, v) + d(v, c_i), the
 * forward distance on G plus the forward distance from c_i on the reversed
 * graph G^T.  Returns -2 if a sum does not fit uint32. */
int orc_roundtrip_table(int64_t n, const int64_t *fw_row_ptr,
                        const int32_t *fw_col, const uint32_t *fw_w,
                        const int64_t *rv_row_ptr, const int32_t *rv_col,
                        const uint32_t *rv_w, int32_t k,
                        const int32_t *sources, uint32_t *table)
{
    uint32_t *rev = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!rev) return -4;
    int rc = 0;
    for (int32_t i = 0; i < k && !rc; ++i) {
        uint32_t *row = table + (size_t)i * n;
        rc = sssp(n, fw_row_ptr, fw_col, fw_w, sources[i], row);
        if (!rc) rc = sssp(n, rv_row_ptr, rv_col, rv_w, sources[i], rev);
        for (int64_t v = 0; v < n && !rc; ++v) {
            if (row[v] == ORC_INF || rev[v] == ORC_INF) { rc = -3; break; }
            uint64_t s = (uint64_t)row[v] + rev[v];
            if (s >= ORC_INF) { rc = -2; break; }
            row[v] = (uint32_t)s;
        }
    }
    free(rev);
    return rc;
}

/* Exact S(v) = sum_u d(v,u) for every v by n SSSPs (eq. (1)).  For round-trip
 * closeness call it on G and on G^T and add the two results. */
int orc_exact_S(int64_t n, const int64_t *row_ptr, const int32_t *col,
                const uint32_t *w, uint64_t *S)
{
    uint32_t *dist = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!dist) return -4;
    int rc = 0;
    for (int64_t v = 0; v < n && !rc; ++v) {
        rc = sssp(n, row_ptr, col, w, (int32_t)v, dist);
        uint64_t s = 0;
        for (int64_t u = 0; u < n && !rc; ++u) {
            if (dist[u] == ORC_INF) rc = -3;
            s += dist[u];
        }
        S[v] = s;
    }
    free(dist);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Estimators from an explicit k x n table of a metric                       */
/* ------------------------------------------------------------------------ */

/* Sample index of each node: sidx[v] = i if v == sources[i], else -1.
 * Returns -1 if a source repeats or is out of range. */
static int sample_index(int64_t n, int32_t k, const int32_t *sources,
                        int32_t *sidx)
{
    for (int64_t v = 0; v < n; ++v) sidx[v] = -1;
    for (int32_t i = 0; i < k; ++i) {
        int32_t c = sources[i];
        if (c < 0 || c >= n || sidx[c] >= 0) return -1;
        sidx[c] = i;
    }
    return 0;
}

/*
 * orc_estimate -- every per-node statistic and estimate from the table.
 *
 * Inputs: table[i*n+v] = d(c_i, v) for a metric (undirected graph distances
 * or round-trip distances); sources[i] = c_i (distinct); eps = a/b, 0<a<=b.
 *
 * Outputs (each may be NULL; with hyb, s_hat and closeness all NULL the
 * estimates are skipped):
 *   pivot[v]    c(v) as a sample index (section 2); own index for v in C
 *   delta[v]    Delta(v) = d(v, c(v)); 0 for v in C
 *   sum[v]      sum_i d(c_i, v) (the sampling accumulator, section 3)
 *   S_samp[i]   exact S(c_i) = sum_v d(c_i, v)
 *   delta_cc[i*k+j]  d(c_i, c_j)
 *   hyb[v*6 + 0..5]  {Hsum, Hnum, HCsum, LCsum, LCnum, LCsumSq} of eq. (4)
 *                    for v not in C; zeros for v in C
 *   s_hat[e*n+v], closeness[e*n+v] for e = 0 sampling, 1 pivoting,
 *                    2 pivoting upper bound, 3 hybrid.
 */
int orc_estimate(int64_t n, int32_t k, const int32_t *sources,
                 const uint32_t *table, uint32_t eps_a, uint32_t eps_b,
                 int32_t *pivot, uint32_t *delta, uint64_t *sum,
                 uint64_t *S_samp, uint32_t *delta_cc, uint64_t *hyb,
                 double *s_hat, double *closeness)
{
    if (n < 2 || k <= 0 || k > n || eps_a == 0 || eps_a > eps_b) return -1;
    int32_t *sidx = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *piv = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    uint32_t *dlt = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint64_t *S = (uint64_t *)malloc((size_t)k * sizeof(uint64_t));
    if (!sidx || !piv || !dlt || !S) {
        free(sidx); free(piv); free(dlt); free(S); return -4;
    }
    if (sample_index(n, k, sources, sidx)) {
        free(sidx); free(piv); free(dlt); free(S); return -1;
    }
#define D(i, v) ((uint64_t)table[(size_t)(i) * (size_t)n + (size_t)(v)])

    /* Exact S(c_i): row sums of the table. */
    for (int32_t i = 0; i < k; ++i) {
        uint64_t s = 0;
        for (int64_t v = 0; v < n; ++v) s += D(i, v);
        S[i] = s;
        if (S_samp) S_samp[i] = s;
    }
    if (delta_cc)
        for (int32_t i = 0; i < k; ++i)
            for (int32_t j = 0; j < k; ++j)
                delta_cc[(size_t)i * k + j] = (uint32_t)D(i, sources[j]);

    /* Pivot: smallest distance, ties to the smallest sample index. */
    for (int64_t v = 0; v < n; ++v) {
        int32_t best = 0;
        for (int32_t i = 1; i < k; ++i)
            if (D(i, v) < D(best, v)) best = i;
        piv[v] = best;
        dlt[v] = (uint32_t)D(best, v);
        if (sidx[v] >= 0) { piv[v] = sidx[v]; dlt[v] = 0; }
        if (pivot) pivot[v] = piv[v];
        if (delta) delta[v] = dlt[v];
    }

    const uint64_t nm1 = (uint64_t)(n - 1);
    /* Only the first-pass statistics asked for: no estimates. */
    const int want_est = hyb || s_hat || closeness;
    for (int64_t j = 0; j < n; ++j) {
        uint64_t sj = 0;
        for (int32_t i = 0; i < k; ++i) sj += D(i, j);
        if (sum) sum[j] = sj;
        if (!want_est) continue;

        double est[4];
        uint64_t h6[6] = {0, 0, 0, 0, 0, 0};
        if (sidx[j] >= 0) {
            /* j in C: exact S(j) for every estimator. */
            double ex = (double)S[sidx[j]];
            est[0] = est[1] = est[2] = est[3] = ex;
        } else {
            const int32_t p = piv[j];
            const uint64_t Dj = dlt[j];
            /* eq. (3) scaled to S: (n-1)/k * sum_i d_ij. */
            est[0] = (double)((u128)nm1 * sj) / (double)k;
            /* pivoting: B(c(j)) -> S(c(j)). */
            est[1] = (double)S[p];
            /* pivoting upper bound: B(c(j)) + Delta(j) -> S(c(j)) + (n-1)Delta. */
            est[2] = (double)((u128)S[p] + (u128)nm1 * Dj);

            /* eq. (4): x lies beyond Delta/eps iff x*a > Delta*b. */
            const u128 thr = (u128)Dj * eps_b;
            uint64_t Hsum = 0, Hnum = 0;
            for (int64_t w = 0; w < n; ++w) {
                if (sidx[w] >= 0) continue;              /* H is in V \ C */
                uint64_t x = D(p, w);                     /* d_{c(j) w} */
                if ((u128)x * eps_a > thr) { Hsum += x; Hnum += 1; }
            }
            uint64_t HCsum = 0, HCnum = 0, LCsum = 0, LCnum = 0, LCsq = 0;
            for (int32_t i = 0; i < k; ++i) {
                uint64_t x = D(p, sources[i]);            /* d_{c(j) c_i} */
                uint64_t dji = D(i, j);                   /* d_{j c_i} */
                if ((u128)x * eps_a > thr) { HCsum += dji; HCnum += 1; }
                else { LCsum += dji; LCnum += 1; LCsq += dji * dji; }
            }
            /* |L(j)| = |V \ {j}| - |H(j)| - |HC(j)|. */
            uint64_t Lnum = nm1 - Hnum - HCnum;
            u128 N = (u128)(Hsum + HCsum) * LCnum + (u128)LCsum * Lnum;
            est[3] = (double)N / (double)LCnum;
            h6[0] = Hsum; h6[1] = Hnum; h6[2] = HCsum;
            h6[3] = LCsum; h6[4] = LCnum; h6[5] = LCsq;
        }
        if (hyb) memcpy(hyb + (size_t)j * 6, h6, sizeof(h6));
        for (int e = 0; e < 4; ++e) {
            if (s_hat) s_hat[(size_t)e * n + j] = est[e];
            if (closeness) closeness[(size_t)e * n + j] = (double)nm1 / est[e];
        }
    }
#undef D
    free(sidx); free(piv); free(dlt); free(S);
    return 0;
}

/* Exact closeness B^-1(v) = (n-1)/S(v) from S (eq. (1)). */
int orc_closeness_from_S(int64_t n, const uint64_t *S, double *closeness)
{
    if (n < 2) return -1;
    for (int64_t v = 0; v < n; ++v)
        closeness[v] = (double)(n - 1) / (double)S[v];
    return 0;
}

/*
 * Error estimate of the hybrid estimate of one node j not in C, for
 * eps = a/b (Algorithm 1's last loop; section 4, eqs. (5) and (6)):
 *
 *   SqErrEst(j) = |L(j)| / |L(j) n C| * var(L(j) n C)
 *               + |H(j)| * SQ(H(j)),
 *
 * var = sample variance of the distances d(c_i, j), c_i in L(j) n C
 * (mean of squares minus square of mean), and SQ(H(j)) = the mean over
 * c_i in HC(j) of (d(c_i, j) - d(c(j), c_i))^2.  When HC(j) is empty the
 * paper falls back to a "suffix" of the sampled nodes farthest from c(j)
 * without giving its size; here it is the single sampled node farthest
 * from c(j) other than c(j) (ties to the smallest index; c(j) itself when
 * k = 1).  Partition as in orc_estimate: x is beyond the threshold iff
 * x*a > Delta(j)*b.  Numerators are exact integers (128-bit), converted
 * once and divided once per term.  Writes the hybrid estimate to *est.
 */
#define D(i, v) ((uint64_t)table[(size_t)(i) * (size_t)n + (size_t)(v)])
static double sqerr_node(int64_t n, int32_t k, const int32_t *sources,
                         const int32_t *sidx, const uint32_t *table, int64_t j, int32_t p,
                         uint64_t Dj, uint32_t a, uint32_t b, double *est)
{
    const uint64_t nm1 = (uint64_t)(n - 1);
    const u128 thr = (u128)Dj * b;
    uint64_t Hsum = 0, Hnum = 0;
    for (int64_t w = 0; w < n; ++w) {
        if (sidx[w] >= 0) continue;
        uint64_t x = D(p, w);
        if ((u128)x * a > thr) { Hsum += x; Hnum += 1; }
    }
    uint64_t HCsum = 0, HCnum = 0, LCsum = 0, LCnum = 0;
    u128 LCsq = 0, HCsqerr = 0;
    int32_t far = p;
    for (int32_t i = 0; i < k; ++i) {
        uint64_t x = D(p, sources[i]);      /* d(c(j), c_i) */
        uint64_t dji = D(i, j);             /* d(c_i, j) */
        if ((u128)x * a > thr) {
            HCsum += dji; HCnum += 1;
            int64_t e = (int64_t)dji - (int64_t)x;
            HCsqerr += (u128)((uint64_t)(e < 0 ? -e : e)) * (uint64_t)(e < 0 ? -e : e);
        } else {
            LCsum += dji; LCnum += 1; LCsq += (u128)dji * dji;
        }
        if (i != p && (far == p || x > D(p, sources[far]))) far = i;
    }
    const uint64_t Lnum = nm1 - Hnum - HCnum;
    u128 N = (u128)(Hsum + HCsum) * LCnum + (u128)LCsum * Lnum;
    *est = (double)N / (double)LCnum;
    /* sampling term: (LCsq*LCnum - LCsum^2) * Lnum / LCnum^3 */
    const u128 var_num = LCsq * LCnum - (u128)LCsum * LCsum;
    const double t1 = (double)(var_num * Lnum) /
                      ((double)LCnum * (double)LCnum * (double)LCnum);
    double t2;
    if (HCnum > 0) {
        t2 = (double)(HCsqerr * Hnum) / (double)HCnum;
    } else {
        int64_t e = (int64_t)D(far, j) - (int64_t)D(p, sources[far]);
        uint64_t ae = (uint64_t)(e < 0 ? -e : e);
        t2 = (double)((u128)ae * ae * Hnum);
    }
    return t1 + t2;
}

/*
 * orc_sqerr -- hybrid estimate and its error estimate SqErrEst for every
 * node (0 for sampled nodes, whose S is exact).  Inputs as orc_estimate.
 */
int orc_sqerr(int64_t n, int32_t k, const int32_t *sources, const uint32_t *table,
              uint32_t eps_a, uint32_t eps_b, double *s_hat, double *sqerr)
{
    if (n < 2 || k <= 0 || k > n || eps_a == 0 || eps_a > eps_b) return -1;
    int32_t *sidx = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!sidx) return -4;
    if (sample_index(n, k, sources, sidx)) { free(sidx); return -1; }
    for (int64_t j = 0; j < n; ++j) {
        if (sidx[j] >= 0) {
            uint64_t s = 0;
            for (int64_t v = 0; v < n; ++v) s += D(sidx[j], v);
            s_hat[j] = (double)s;
            sqerr[j] = 0.0;
            continue;
        }
        int32_t p = 0;
        for (int32_t i = 1; i < k; ++i)
            if (D(i, j) < D(p, j)) p = i;
        sqerr[j] = sqerr_node(n, k, sources, sidx, table, j, p, D(p, j), eps_a, eps_b,
                              &s_hat[j]);
    }
    free(sidx);
    return 0;
}

/*
 * orc_adaptive -- the adaptive hybrid ("Hyb.-ad", section 6): for every
 * node not in C, the hybrid estimate under each eps = as[e]/bs[e] of the
 * list, keeping the one with the smallest SqErrEst (ties to the earlier
 * entry).  choice[j] is that entry's position; -1 for sampled nodes, which
 * get their exact S and error 0.
 */
int orc_adaptive(int64_t n, int32_t k, const int32_t *sources, const uint32_t *table,
                 int32_t ne, const uint32_t *as, const uint32_t *bs, double *s_hat,
                 double *sqerr, int32_t *choice)
{
    if (n < 2 || k <= 0 || k > n || ne <= 0) return -1;
    for (int32_t e = 0; e < ne; ++e)
        if (as[e] == 0 || as[e] > bs[e]) return -1;
    int32_t *sidx = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!sidx) return -4;
    if (sample_index(n, k, sources, sidx)) { free(sidx); return -1; }
    for (int64_t j = 0; j < n; ++j) {
        if (sidx[j] >= 0) {
            uint64_t s = 0;
            for (int64_t v = 0; v < n; ++v) s += D(sidx[j], v);
            s_hat[j] = (double)s;
            sqerr[j] = 0.0;
            choice[j] = -1;
            continue;
        }
        int32_t p = 0;
        for (int32_t i = 1; i < k; ++i)
            if (D(i, j) < D(p, j)) p = i;
        for (int32_t e = 0; e < ne; ++e) {
            double est;
            double se = sqerr_node(n, k, sources, sidx, table, j, p, D(p, j), as[e], bs[e],
                                   &est);
            if (e == 0 || se < sqerr[j]) { sqerr[j] = se; s_hat[j] = est; choice[j] = e; }
        }
    }
    free(sidx);
    return 0;
}

#undef D

/*
 * Streaming form of the sampling and pivoting statistics (section 3, second
 * paragraph): one SSSP per sampled node, each scanned node v adds d to
 * sum[v] and updates the running minimum Delta(v) / pivot c(v) (strict "<",
 * so the smallest index wins ties because sources run in index order).
 * Needs O(1) state per node -- no k x n table.  Used to time the CPU
 * baseline; must agree with orc_estimate.
 */
int orc_streaming_pass(int64_t n, const int64_t *row_ptr, const int32_t *col,
                       const uint32_t *w, int32_t k, const int32_t *sources,
                       uint64_t *sum, int32_t *pivot, uint32_t *delta,
                       uint64_t *S_samp)
{
    if (n < 2 || k <= 0 || k > n) return -1;
    uint32_t *dist = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!dist) return -4;
    for (int64_t v = 0; v < n; ++v) { sum[v] = 0; pivot[v] = -1; delta[v] = ORC_INF; }
    int rc = 0;
    for (int32_t i = 0; i < k && !rc; ++i) {
        rc = sssp(n, row_ptr, col, w, sources[i], dist);
        uint64_t s = 0;
        for (int64_t v = 0; v < n && !rc; ++v) {
            uint32_t d = dist[v];
            if (d == ORC_INF) { rc = -3; break; }
            sum[v] += d;
            s += d;
            if (d < delta[v]) { delta[v] = d; pivot[v] = i; }
        }
        if (S_samp) S_samp[i] = s;
    }
    free(dist);
    return rc;
}
