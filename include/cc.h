/*
 * cc.h -- C ABI of the GB300 (sm_103a) library for all-nodes classic
 * closeness estimation after Cohen, Delling, Pajor and Werneck, "Computing
 * Classic Closeness Centrality, at Scale" (2014).
 *
 * Problem (eq. (1)): for a connected undirected graph G = (V, E) with n = |V|
 * nodes, B^-1(v) = (n-1) / S(v) with S(v) = sum_u d_vu.  For a strongly
 * connected directed graph the round-trip distance d_uv + d_vu is used
 * instead (section 6.1).
 *
 * Method (sections 2 and 3): choose a uniform sample C = (c_0 .. c_{k-1}) of
 * k nodes, run one shortest-path traversal from every sampled node (BFS when
 * unweighted, SSSP with uint32 arc lengths otherwise) and reduce the
 * distances on the fly into per-node statistics, never storing the k x n
 * distance matrix.  From them the library forms, for every node, the sampling
 * estimate (eq. (3)), the pivoting estimate B(c(v)), the pivoting upper bound
 * B(c(v)) + Delta(v) and the hybrid estimate (eq. (4)).  Further entry
 * points give the hybrid's error estimate and the adaptive hybrid
 * (sections 4, 6), node-weighted closeness (section 5), outbound / inbound
 * estimates of general directed graphs (section 6.2), batches of graphs in
 * one launch and a serving loop.
 *
 * Conventions for every entry point:
 *   - returns CC_OK (0) or a negative CC_ERR_* code; no exception crosses the
 *     ABI; cc_strerror() names a code;
 *   - host pointers unless stated; the library copies every input it keeps
 *     and never takes ownership of caller memory;
 *   - calls are synchronous: when one returns, its outputs are written;
 *   - a graph handle may be used by one thread at a time.
 *
 * Readings of the paper fixed by this interface:
 *   - eps is the rational eps_num / eps_den with 0 < eps_num <= eps_den;
 *     membership of H and HC (section 2, eq. (4): beyond Delta/eps from the
 *     pivot) is tested exactly, in integers, as d * eps_num > Delta * eps_den;
 *   - the pivot c(v) is the sampled node at minimum distance, ties to the
 *     smallest sample index; a sampled node is its own pivot;
 *   - every estimator returns the exact S(v) for v in C;
 *   - FP64 results: the integer numerator is formed in 128 bits, converted
 *     to double once and divided once.
 */
#ifndef CC_GB300_H
#define CC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define CC_OK 0
#define CC_ERR_ARG (-1)          /* bad argument (null, range, duplicate) */
#define CC_ERR_GRAPH (-2)        /* malformed graph (ids out of range, n<2) */
#define CC_ERR_DISCONNECTED (-3) /* closeness undefined: not (strongly) connected */
#define CC_ERR_OOM (-4)          /* device or host allocation failed */
#define CC_ERR_TIMEOUT (-5)      /* a bounded device-side wait ran out */
#define CC_ERR_CUDA (-6)         /* a CUDA runtime call failed */
#define CC_ERR_TOO_LARGE (-7)    /* size beyond a documented limit */
#define CC_ERR_NO_DEVICE (-8)    /* no usable CUDA device */

/* Maximum sample size: k sources are packed 64 per uint64 word, at most 32
 * words per node. */
#define CC_MAX_K 2048

/* ---- graphs ------------------------------------------------------------ */
typedef struct cc_graph *cc_graph_t;

/*
 * cc_graph_from_edges -- build the device-resident graph the estimators run
 * on (the "graph to CSR" step; section 7 counts this preprocessing in its
 * times).
 *   n              number of node ids; every src[e], dst[e] must be < n
 *   m              number of edges in src/dst (and w)
 *   src, dst       uint32[m] edge endpoints (host)
 *   w              uint32[m] arc lengths >= 1, or NULL for unweighted
 *   directed       0: each edge is undirected (arcs both ways);
 *                  1: each edge is the arc src -> dst
 *   keep_component 1: keep only the largest connected component (largest
 *                  strongly connected component when directed; ties to the
 *                  component holding the smallest id); 0: keep every node
 *   out            receives the handle
 *   old_id_out     optional int32[n] (caller-owned): old_id_out[v'] = the
 *                  original id of kept node v' for v' < n' (the kept count,
 *                  from cc_graph_info); entries beyond n' are untouched
 * Self-loops are dropped, parallel arcs merged keeping the smallest length,
 * kept nodes renumbered 0..n'-1 in increasing original id, adjacency lists
 * sorted by neighbour.  Errors: CC_ERR_ARG, CC_ERR_GRAPH, CC_ERR_OOM,
 * CC_ERR_CUDA, CC_ERR_TOO_LARGE (more than 2^31-1 arcs or nodes).
 */
int cc_graph_from_edges(int64_t n, int64_t m, const uint32_t *src,
                        const uint32_t *dst, const uint32_t *w, int directed,
                        int keep_component, cc_graph_t *out,
                        int32_t *old_id_out);

/* Same as cc_graph_from_edges with the arcs given as a CSR
 * (row_ptr int64[n+1], col int32[row_ptr[n]], w uint32[row_ptr[n]] or NULL):
 * arc e of row u is u -> col[e].  For undirected graphs each listed arc
 * also gives its reverse. */
int cc_graph_load_csr(int64_t n, const int64_t *row_ptr, const int32_t *col,
                      const uint32_t *w, int directed, int keep_component,
                      cc_graph_t *out, int32_t *old_id_out);

/* Release the handle and all device memory it owns. */
int cc_graph_free(cc_graph_t g);

/* Sizes of a built graph: n kept nodes, arcs (CSR entries: 2m undirected,
 * m directed), directed and weighted flags.  Any pointer may be NULL. */
int cc_graph_info(cc_graph_t g, int64_t *n, int64_t *arcs, int *directed,
                  int *weighted);

/* Copy the built CSR back to caller host buffers (row_ptr int64[n+1],
 * col int32[arcs], w uint32[arcs] or NULL).  With reverse = 1 the CSR of
 * the reversed graph (directed graphs only). */
int cc_graph_copy_csr(cc_graph_t g, int reverse, int64_t *row_ptr,
                      int32_t *col, uint32_t *w);

/* ---- sample ---------------------------------------------------------- */
/*
 * cc_sample_choose -- uniform sample of k distinct nodes (section 2: k
 * nodes drawn uniformly without replacement; Algorithm 1, first step).
 * Node v gets the key splitmix64(seed, v) =
 * mix(seed + (v+1) * 0x9E3779B97F4A7C15) with the splitmix64 output
 * function mix (Steele, Lea, Flood 2014); the sample is the k nodes with the
 * smallest (key, v), in that order (bottom-k sampling, uniform without
 * replacement).  sample_out int32[k] (host).  Computed on the
 * device.  Errors: CC_ERR_ARG (k < 1, k > n or k > CC_MAX_K).
 */
int cc_sample_choose(cc_graph_t g, int32_t k, uint64_t seed,
                     int32_t *sample_out);

/* ---- estimation -------------------------------------------------------- */
#define CC_EST_SAMPLING 0     /* eq. (3): (n-1)/k * sum_i d(c_i, v)   */
#define CC_EST_PIVOTING 1     /* S(c(v))                                */
#define CC_EST_PIVOT_UPPER 2  /* S(c(v)) + (n-1) Delta(v)               */
#define CC_EST_HYBRID 3       /* eq. (4)                                */
#define CC_NUM_EST 4

/* Output pointers: host memory unless cc_opts.device_outputs = 1 (then
 * device pointers on the current device).  Every pointer may be NULL. */
typedef struct {
    double *s_hat[CC_NUM_EST];     /* n each: estimate of S(v)            */
    double *closeness[CC_NUM_EST]; /* n each: (n-1) / s_hat               */
    int32_t *pivot;                /* n: c(v) as a sample index           */
    uint32_t *delta;               /* n: Delta(v) = d(v, c(v))            */
    uint64_t *sample_sum;          /* n: sum_i d(c_i, v)                  */
    uint64_t *hyb_int;             /* n x 6: Hsum Hnum HCsum LCsum LCnum
                                      LCsumSq of eq. (4); zeros for v in C */
    uint64_t *S_sampled;           /* k: exact S(c_i)                     */
    uint32_t *delta_cc;            /* k x k: d(c_i, c_j), row i           */
    double *sq_err;                /* n: SqErrEst of the hybrid estimate
                                      (Algorithm 1's last loop, section 4):
                                      |L| var(L n C)/|L n C| + |H| * mean
                                      over HC of (d(c_i,v) - d(c(v),c_i))^2;
                                      when HC(v) is empty the sampled node
                                      farthest from c(v) stands in for it;
                                      0 for v in C.  Needs want_hybrid; asking
                                      for it may add the second pass.      */
} cc_out;

typedef struct {
    uint32_t eps_num, eps_den; /* hybrid eps = num/den; 0 < num <= den    */
    int32_t want_hybrid;       /* 1: run the second traversal when eq. (4)
                                  needs it; 0: skip (hybrid outputs unset) */
    int32_t roundtrip;         /* directed graphs: 1 = round-trip distances
                                  (section 6.1); required for directed     */
    int32_t device_outputs;    /* 1: cc_out pointers are device pointers   */
    void *stream;              /* cudaStream_t, NULL = legacy default      */
} cc_opts;

/* Fill defaults: eps = 1/round(sqrt(k)) (section 7: eps = sqrt(1/k)),
 * want_hybrid = 1, roundtrip = 0, host outputs, default stream. */
void cc_opts_default(cc_opts *o, int32_t k);

/*
 * cc_estimate -- all-nodes estimates from one seeded sample.
 *   sample  int32[k] distinct node ids (host), e.g. from cc_sample_choose;
 *           sample index i fixes the bit position and the pivot tie-break.
 * Runs the k traversals as one bit-packed multi-source pass (pass 1: sums,
 * pivots, Delta, d(c_i, c_j), per-source distance histograms) and, when the
 * hybrid needs per-node thresholds below the largest sampled distance, a
 * second pass with the per-node L(v) masks (section 3, Algorithm 1).
 * Errors: CC_ERR_ARG, CC_ERR_DISCONNECTED, CC_ERR_OOM, CC_ERR_TIMEOUT,
 * CC_ERR_CUDA, CC_ERR_TOO_LARGE (a distance >= 2^32-1).
 */
int cc_estimate(cc_graph_t g, const int32_t *sample, int32_t k,
                const cc_opts *opts, cc_out *out);

/*
 * cc_estimate_adaptive -- the adaptive hybrid ("Hyb.-ad", section 6; the
 * error estimate of section 4): one first traversal pass, then for each
 * eps = eps_num[e]/eps_den[e] of the list the hybrid estimate of eq. (4)
 * and its SqErrEst (see cc_out.sq_err); every node keeps the estimate with
 * the smallest SqErrEst (ties to the earlier entry).  eps_num = eps_den =
 * NULL selects the paper's list 0.001, 0.025, 0.05, 0.1, 0.2, 0.5, 0.99
 * (n_eps ignored).  Outputs, n each, host or device per
 * opts->device_outputs, any may be NULL: s_hat (sampled nodes: exact S),
 * closeness (n-1)/s_hat, sq_err (0 for sampled nodes), choice (the entry
 * used; -1 for sampled nodes).  opts->eps_* and want_hybrid are ignored;
 * roundtrip must match the graph.  Each entry costs the ε-dependent part of
 * cc_estimate again: thresholds and, where some node needs it, the second
 * traversal pass.  Errors: as cc_estimate; CC_ERR_ARG for n_eps outside
 * 1..64 or an entry with eps_num = 0 or eps_num > eps_den.
 */
int cc_estimate_adaptive(cc_graph_t g, const int32_t *sample, int32_t k,
                         const cc_opts *opts, int32_t n_eps, const uint32_t *eps_num,
                         const uint32_t *eps_den, double *s_hat, double *closeness,
                         double *sq_err, int32_t *choice);

/* ---- node weights -------------------------------------------------------- */
/*
 * Node-weighted closeness (section 5, "Weighted Centrality"; its
 * modification of Algorithm 1).  With node weights beta(v) >= 0,
 * S_beta(v) = sum over u != v of beta(u) d(v, u) and the weighted closeness
 * is (B - beta(v)) / S_beta(v), B the sum of all weights.
 *
 * cc_graph_set_node_weights -- attach beta (uint32[n], host, indexed by the
 * graph's node numbering; NULL detaches).  The library copies it.  Errors:
 * CC_ERR_ARG (null handle), CC_ERR_TOO_LARGE (B >= 2^40), CC_ERR_OOM,
 * CC_ERR_CUDA.
 */
int cc_graph_set_node_weights(cc_graph_t g, const uint32_t *beta);

/*
 * cc_sample_varopt -- weighted sample of exactly k nodes (section 5): node v
 * is in it with probability min(1, beta(v)/tau), tau the threshold with
 * sum over v of min(1, beta(v)/tau) = k, written to tau_out[0] / tau_out[1]
 * as an exact fraction (numerator, denominator).  The draw is systematic
 * sampling with unequal probabilities along the order of splitmix64 keys
 * (output number v of stream `seed` for node v, the keys of
 * cc_sample_choose; ties by id), with offset floor(x * tau_num / 2^64),
 * x = output number n of the stream.  sample_out int32[k] (host) lists the
 * sampled nodes in that order.  Errors: CC_ERR_ARG (no weights attached,
 * k < 1 or fewer than k positive weights), CC_ERR_OOM, CC_ERR_CUDA.
 */
int cc_sample_varopt(cc_graph_t g, int32_t k, uint64_t seed, int32_t *sample_out,
                     uint64_t *tau_out);

typedef struct {
    double *s_hat[2];     /* n each: estimate of S_beta(v); [0] sampling
                             (inverse probability: sum over c in C of
                             max(tau, beta(c)) d(c, v)), [1] hybrid; sampled
                             nodes get their exact S_beta                   */
    double *closeness[2]; /* n each: (B - beta(v)) / s_hat                  */
    uint64_t *S_sampled;  /* k: exact S_beta(c_i)                           */
} cc_wout;

/*
 * cc_estimate_node_weighted -- node-weighted estimates from a weighted
 * sample (e.g. cc_sample_varopt's) and its threshold tau = tau[0]/tau[1].
 * Hybrid, for v not sampled with pivot p = c(v) and Delta = d(p, v) (x is
 * beyond when x * eps_num > Delta * eps_den): each non-sampled w beyond from
 * p counts beta(w) d(p, w), each sampled c_i with d(p, c_i) beyond counts
 * beta(c_i) d(c_i, v), each other sampled node max(tau, beta(c_i)) d(c_i, v).
 * Every estimate is an integer numerator over tau[1] divided once in FP64.
 * Runs the sources in chunks of shortest-path rows for every graph kind
 * (a second sweep for the hybrid when opts->want_hybrid).  opts: eps,
 * want_hybrid, roundtrip (must match the graph), device_outputs, stream.
 * Errors: CC_ERR_ARG (no weights attached, bad sample or tau = 0/x),
 * CC_ERR_DISCONNECTED, CC_ERR_OOM, CC_ERR_TIMEOUT, CC_ERR_CUDA,
 * CC_ERR_TOO_LARGE (B x largest distance >= 2^63, or the adjusted weights'
 * sum x tau[1] x largest distance >= 2^64).
 */
int cc_estimate_node_weighted(cc_graph_t g, const int32_t *sample, int32_t k,
                              const uint64_t *tau, const cc_opts *opts, cc_wout *out);

/* ---- general directed graphs ---------------------------------------------- */
/*
 * cc_reach_estimate -- outbound / inbound estimates of general (not
 * necessarily strongly connected) directed graphs (section 6.2, Algorithm
 * 4).  With the nodes in a seeded random order (increasing splitmix64
 * output number v of stream `seed`, ties by id -- the keys of
 * cc_sample_choose), node v's sample is the k nodes of smallest rank among
 * R(v), the nodes other than v that v reaches (inbound != 0: that reach v).
 *   avg_dist  double[n]: average distance to the sample (0 when R(v) is
 *             empty) -- the estimate of S(v)/|R(v)|, whose inverse is the
 *             outbound (inbound) centrality
 *   reach     double[n]: |R(v)| when it is below k, else the bottom-k
 *             estimate 1 + (k-1)(n-2)/(T(v)-1) (1 when k = 1)
 *   count     int32[n]: samples taken, min(k, |R(v)|)
 *   dist_sum  uint64[n]: sum of the sample's distances
 *   T         int64[n]: rank position (1-based, not counting v) of the k-th
 *             sample; 0 when count < k
 * Outputs are host arrays, any may be NULL.  Runs one cooperative launch
 * over the order in groups of 512 sources by default (CC_PARAM_REACH_WORDS):
 * bit-packed searches on G^T (outbound) or G (inbound) that skip nodes
 * already holding k + 1 nodes of smaller rank (themselves included);
 * breadth-first on unit lengths,
 * label-correcting shortest paths with arc lengths (distances must stay
 * below 2^32 - 1).  Errors: CC_ERR_ARG (k < 1), CC_ERR_OOM, CC_ERR_CUDA,
 * CC_ERR_TIMEOUT (a bounded device-side wait ran out).
 */
int cc_reach_estimate(cc_graph_t g, int32_t k, uint64_t seed, int32_t inbound, void *stream,
                      double *avg_dist, double *reach, int32_t *count, uint64_t *dist_sum,
                      int64_t *T);

/* ---- exact values and single-source reference ---------------------------- */
/*
 * cc_exact -- exact S(v) and B^-1(v) = (n-1)/S(v) for every node (eq. (1))
 * by traversals from every node, packed 64 per word.  Meant for small
 * graphs (the cost is n traversals).  closeness double[n], S uint64[n] (host,
 * either may be NULL).  Errors as cc_estimate.
 */
int cc_exact(cc_graph_t g, double *closeness, uint64_t *S);

/*
 * cc_sampling_sums_single -- reference form of the sampling pass: k
 * separate single-source traversals, one launch per sampled node, each adding
 * its distances to sum[v] (section 3, second paragraph).  Same results as
 * cc_estimate's sample_sum; kept to measure what bit-packing k sources per
 * traversal buys.  sum uint64[n] (host), S_sampled uint64[k] (host, may be
 * NULL).
 */
int cc_sampling_sums_single(cc_graph_t g, const int32_t *sample, int32_t k,
                            uint64_t *sum, uint64_t *S_sampled);

/*
 * cc_sampling_pivots_noalloc -- the first traversal pass of cc_estimate
 * (per-node sum of distances to the sample, pivot, Delta, and the exact S of
 * every sampled node) for callers that cannot allocate device memory, e.g.
 * code running inside a framework whose memory pool owns the device, or under
 * a memory budget where an allocation could fail or synchronise the device at
 * the wrong moment.  The paper has no counterpart: it is a deployment variant
 * of the same computation.
 *   n            nodes; d_row_ptr int64[n+1] and d_col int32[row_ptr[n]] are
 *                a connected undirected graph in device memory (each edge
 *                listed both ways, e.g. as returned by cc_graph_copy_csr).
 *                The device checks that the row offsets ascend within the
 *                arcs, that every column is a node id and that every node
 *                has as many arcs in as out (CC_ERR_GRAPH otherwise).  The
 *                last is only a necessary condition of symmetry: a CSR that
 *                passes it without being symmetric gives undefined results
 *   sample, k    host int32[k], distinct node ids (CC_ERR_ARG otherwise)
 *   outputs      device memory owned by the caller: d_sample_sum uint64[n],
 *                d_pivot int32[n], d_delta uint32[n], d_S_sampled uint64[k]
 *   stream       cudaStream_t or NULL
 * Allocates nothing: all working memory lives in one fixed 32 MiB device
 * array inside the library, present on every GPU that loads the library until
 * the process exits.  A call that needs more -- about 4*n*W*8 + 52*n +
 * 4*k*k + 8192*k bytes with W = ceil(k/64) rounded up to a power of two --
 * returns CC_ERR_TOO_LARGE before touching the device.  A traversal deeper
 * than 2047 levels (the array's distance histogram) is found only after the
 * pass: the call then returns CC_ERR_TOO_LARGE with the outputs partly
 * written and undefined.
 * The first call on a device looks up that array's device address (once per
 * device, with the device current); make that first call before any stream
 * capture.  Every call reuses the array and clears what it needs; calls that
 * overlap on the GPU race on it and must not be issued.  Synchronous on
 * `stream`.
 */
int cc_sampling_pivots_noalloc(int64_t n, const int64_t *d_row_ptr,
                               const int32_t *d_col, const int32_t *sample,
                               int32_t k, uint64_t *d_sample_sum,
                               int32_t *d_pivot, uint32_t *d_delta,
                               uint64_t *d_S_sampled, void *stream);

/* ---- batches: many graphs in one persistent launch ------------------------- */
typedef struct cc_batch *cc_batch_t;

/*
 * cc_batch_create -- prepare all-nodes estimates (sections 2-3, every
 * estimator) for ngraphs resident unweighted undirected graphs at once.
 *   graphs[i]      handles (must outlive the batch)
 *   samples[i]     host int32[ks[i]] distinct node ids of graph i
 *   ks[i]          1 <= k <= 512
 *   eps_num/den    per-graph hybrid eps (NULL: 1/round(sqrt(k)))
 *   autotune       1: time every graph alone under the direction switches
 *                  alpha in {default, 2, 4, 8, 14} and keep the fastest per
 *                  graph; per word-width class, model every team count and
 *                  two block shapes (the kernel's full residency per SM and
 *                  half of it) and time the six best plans;
 *                  0: default alpha, plan from CSR sizes only
 * The graphs fall into classes by their word width W (1, 2, 4 or 8 64-bit
 * words per node).  A run is one cooperative launch per class, specialised
 * for its W and covering the GPU, the classes one after another: the CTAs
 * of a class form equal teams, each team estimating its graphs one after
 * another with team-wide bounded barriers.  The hybrid is classified during
 * the first traversal (as cc_estimate's one-pass form) when the graph's
 * band rows could be allocated.  The launches (and their memsets) are
 * captured in a CUDA graph on the first run when the runtime allows it.
 * Device memory for every graph's state and results is owned by the batch.
 * Errors: CC_ERR_ARG, CC_ERR_OOM, CC_ERR_CUDA.
 */
int cc_batch_create(int32_t ngraphs, const cc_graph_t *graphs,
                    const int32_t *const *samples, const int32_t *ks,
                    const uint32_t *eps_num, const uint32_t *eps_den,
                    int32_t autotune, cc_batch_t *out);

/* One batched run on `stream` (cudaStream_t or NULL); synchronous.  Returns
 * the first per-graph error (CC_ERR_DISCONNECTED, CC_ERR_TOO_LARGE when a
 * graph needs more than 8191 levels, CC_ERR_TIMEOUT) or CC_OK. */
int cc_batch_run(cc_batch_t b, void *stream);

/* Copy graph i's results of the last run into `out` (host pointers, or
 * device pointers with device_outputs = 1); same fields as cc_estimate. */
int cc_batch_result(cc_batch_t b, int32_t i, const cc_out *out,
                    int32_t device_outputs);

/* Plan and timing of the last run: teams over all classes, CTAs of the
 * largest class launch, device time of the last run in ms (CUDA events
 * around the launches), whether the run replayed a captured CUDA graph.
 * Any pointer may be NULL. */
int cc_batch_info(cc_batch_t b, int32_t *teams, int32_t *grid, double *last_ms,
                  int32_t *graph_captured);

/* Graph i's place in the plan: its word width, the direction switch it
 * runs with, its team within its class, the class's team count, CTAs and
 * resident CTAs per SM, and whether its tuning came from the autotune
 * cache (1) or was measured (0).  Any pointer may be NULL. */
int cc_batch_plan(cc_batch_t b, int32_t i, int32_t *words, int32_t *alpha, int32_t *team,
                  int32_t *class_teams, int32_t *class_ctas, int32_t *ctas_per_sm,
                  int32_t *from_cache);

/* Autotune cache of cc_batch_create (autotune = 1): a file of one JSON
 * object per line, keyed by the GPU's name, n, arcs, k and the counts of
 * the degree classes (nodes of <= 4, <= 32, <= 128 and more arcs), holding
 * the direction switch that ran the graph fastest alone, that time and the
 * level count.  A graph whose key is in the file skips its timing; the
 * others are timed and appended.  path = NULL or "" turns the cache off
 * (the default).  Process-wide. */
int cc_batch_tune_cache(const char *path);

int cc_batch_free(cc_batch_t b);

/* ---- serving ------------------------------------------------------------------ */
typedef struct cc_server *cc_server_t;

/*
 * cc_server_create -- serve all-nodes estimates (section 2 estimators) over a
 * pool of resident graphs with continuous batching.
 *   graphs        handles kept resident (must outlive the server)
 *   slots         1..64 concurrent requests; each slot has a worker thread,
 *                 a CUDA stream and its own workspace, and its launches use
 *                 at most 1/slots of the GPU's CTAs so that slots overlap
 *   hbm_budget    bytes of device memory the running requests may use
 *                 (0: half of the free memory at creation)
 * A submitted request waits, first come first served, until a slot is free
 * and its footprint fits in the budget left by the running ones.  The first
 * pass of every completed request stays resident (within the budget, least
 * recently used evicted first): a later request for the same graph, k and
 * seed, with any estimator or eps, skips it.
 */
int cc_server_create(int32_t ngraphs, const cc_graph_t *graphs, int32_t slots,
                     uint64_t hbm_budget, cc_server_t *out);

/* Queue a request: graph index, estimator (CC_EST_*), k, sample seed (the
 * sample is cc_sample_choose's), eps = eps_num/eps_den.  Non-blocking;
 * returns its id.  CC_ERR_TOO_LARGE when it could never fit the budget. */
int cc_server_submit(cc_server_t s, int32_t graph, int32_t estimator, int32_t k,
                     uint64_t seed, uint32_t eps_num, uint32_t eps_den,
                     int64_t *request_id);

/* Wait up to timeout_ms for a request: CC_OK when done, its error code when
 * it failed, CC_ERR_TIMEOUT when still waiting or running. */
int cc_server_wait(cc_server_t s, int64_t request_id, int32_t timeout_ms);

/* Copy a finished request's results (host arrays of the graph's n nodes,
 * each may be NULL: the requested estimator's S estimate and closeness,
 * pivot, Delta, sum of distances to the sample) and its latency from
 * submission to completion in ms; releases the request. */
int cc_server_result(cc_server_t s, int64_t request_id, double *s_hat,
                     double *closeness, int32_t *pivot, uint32_t *delta,
                     uint64_t *sample_sum, double *latency_ms);

/* Latency statistics over the completed requests (ms, submission to
 * completion) and the largest number of requests that ran at once. */
int cc_server_stats(cc_server_t s, int64_t *completed, double *p50_ms,
                    double *p99_ms, double *mean_ms, int32_t *peak_running);

/* Resident sampled state: requests that found their (graph, k, seed)
 * first pass resident (hits) or ran it (misses), the states held and the
 * device bytes the idle ones hold.  Any pointer may be NULL. */
int cc_server_cache_stats(cc_server_t s, int64_t *hits, int64_t *misses, int32_t *states,
                          uint64_t *resident_bytes);

/* Drain the queue, stop the workers and release the server. */
int cc_server_free(cc_server_t s);

/* ---- tuning ---------------------------------------------------------------- */
/* Direction switch of the breadth-first traversal of one graph (0 restores
 * the default: 6 when the sample fits one 64-bit word and the mean degree
 * is at least 8, else 14): a level
 * runs top-down while (CSR entries of the frontier) * alpha < (CSR entries
 * of the nodes some source has not reached yet), bottom-up otherwise.
 * Results do not depend on it, only the time. */
int cc_set_tuning(cc_graph_t g, int32_t alpha);

/* Parameters of a graph's estimates (cc_set_param); results never depend
 * on them, only the time.
 *   CC_PARAM_ALPHA            the direction switch of cc_set_tuning (0:
 *                             default)
 *   CC_PARAM_HYBRID_ONE_PASS  1 (default): the bit-packed path classifies
 *                             each arriving bit for the hybrid during the
 *                             first pass -- by the triangle inequality,
 *                             d(c(v), c_i) lies within d(c_i, v) -+ Delta(v)
 *                             (section 3) -- keeping only the undecided
 *                             ones (a byte per node and source) to resolve
 *                             once the distances between sampled nodes are
 *                             known, so no second traversal runs unless a
 *                             band offset exceeds a byte, the error estimate
 *                             is asked for, or the rows do not fit a third
 *                             of the free memory; 0: always the two-pass
 *                             form
 *   CC_PARAM_SSSP_DELTA       bucket width of the shortest-path rounds with
 *                             arc lengths (delta-stepping with a near and a
 *                             far queue: labels below the threshold relax
 *                             in rounds, the others wait until the near
 *                             queue empties and the threshold moves on);
 *                             0 restores the default (96 mean arc
 *                             lengths), a negative value relaxes every
 *                             label at once (plain label-correcting
 *                             rounds)
 *   CC_PARAM_REACH_WORDS      words per node of cc_reach_estimate's groups
 *                             (1, 2, 4, 8 or 16: groups of 64 x that many
 *                             sources searched together); 0 restores the
 *                             default
 *   CC_PARAM_ESTIMATE_GRAPH   1 (default): a bit-packed cc_estimate called
 *                             again with the same k, options and output
 *                             buffers (and no device buffer of the library
 *                             resized since) captures its device work --
 *                             every kernel and memset between the sample
 *                             upload and the output copies -- in a CUDA
 *                             graph once and replays it on later such
 *                             calls (one launch instead of about twenty);
 *                             0: always launched one by one */
#define CC_PARAM_ALPHA 0
#define CC_PARAM_HYBRID_ONE_PASS 1
#define CC_PARAM_SSSP_DELTA 2
#define CC_PARAM_REACH_WORDS 3
#define CC_PARAM_ESTIMATE_GRAPH 4
int cc_set_param(cc_graph_t g, int32_t param, int32_t value);

/* ---- diagnostics --------------------------------------------------------- */
/* Counters of the last traversal pass run on g: levels, top-down and
 * bottom-up levels, CSR entries examined and frontier words gathered.
 * Any pointer may be NULL. */
int cc_last_pass_stats(cc_graph_t g, int64_t *levels, int64_t *td_levels,
                       int64_t *bu_levels, int64_t *edges_examined,
                       int64_t *words_gathered);

/* Phases of a bit-packed traversal pass, for cc_last_pass_phases:
 * state clearing and seeding (level 0); top-down queue building, pushes and
 * finalisation of the touched nodes; bottom-up rebuild of the active light
 * list, light, medium and heavy nodes, finalisation of the heavy nodes; and
 * waiting in the grid barrier between them. */
enum {
    CC_PH_INIT = 0,
    CC_PH_TD_QUEUE = 1,
    CC_PH_TD_PUSH = 2,
    CC_PH_TD_FINAL = 3,
    CC_PH_BU_REBUILD = 4,
    CC_PH_BU_LIGHT = 5,
    CC_PH_BU_MEDIUM = 6,
    CC_PH_BU_HEAVY = 7,
    CC_PH_BU_FINAL = 8,
    CC_PH_BARRIER = 9,
    CC_NUM_PHASES = 10
};

/* Warp time by phase of the last bit-packed traversal pass on g (tracing;
 * the paper has no counterpart): warp_cycles[p] (caller-owned, CC_NUM_PHASES
 * entries) receives the SM clock cycles summed over all warps spent in phase
 * p.  Only the shares are meaningful.  Zero after a weighted pass. */
int cc_last_pass_phases(cc_graph_t g, int64_t *warp_cycles);

/* Per-level trace of the last traversal pass on g (levels 1 .. D, at most
 * max_levels and at most 64): device time of each level in ns (global timer
 * on the device), whether it ran top-down (1) or bottom-up (0), the frontier
 * size it started from, the CSR entries of that frontier and the frontier
 * words it gathered.  Entry 0 is zero; any pointer may be NULL.  Returns the
 * number of entries written (D + 1, capped) or a negative CC_ERR_* code. */
int cc_last_pass_trace(cc_graph_t g, int32_t max_levels, int64_t *level_ns,
                       int32_t *top_down, int64_t *frontier,
                       int64_t *frontier_arcs, int64_t *words);

/* Traversal kernel launches of the last cc_estimate / cc_exact /
 * cc_sampling_sums_single call on g: their number, their summed device time
 * in ms (CUDA events recorded on the launching stream around each launch)
 * and the algorithmic bytes they moved under the library's roofline model
 * (frontier words gathered x 8 B, CSR entries x 4 B, three W-word state
 * arrays per node and level, row offsets of top-down levels, per-node
 * results), and the number of all library kernels the call launched.
 * Any pointer may be NULL. */
int cc_last_call_timing(cc_graph_t g, int32_t *launches, double *kernel_ms,
                        double *alg_bytes, int32_t *all_kernels);

/* *replayed = 1 when the last cc_estimate on g replayed its captured CUDA
 * graph (CC_PARAM_ESTIMATE_GRAPH), else 0. */
int cc_last_call_graph(cc_graph_t g, int32_t *replayed);

/* Run the device-side bounded wait on a barrier that can never complete
 * (a team larger than the blocks launched) with the given limit; returns
 * CC_ERR_TIMEOUT when the wait gives up as designed. */
int cc_selftest_barrier_timeout(uint64_t timeout_ns);

const char *cc_strerror(int code);
/* With the environment variable CC_DEBUG set, every CUDA runtime call that
 * fails inside the library (before it is reported as CC_ERR_CUDA) is named
 * on stderr with its source position. */

#ifdef __cplusplus
}
#endif
#endif /* CC_GB300_H */
