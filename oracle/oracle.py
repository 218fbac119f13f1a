"""Python side of the CPU oracle (TEST INFRASTRUCTURE ONLY).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg
may import this module.  It never imports the GPU package and the GPU package
never imports it; the two share only the seeded edge-list generators.

Pieces:
  * graph building from an edge list with numpy/scipy primitives (a sort for
    de-duplication, scipy's connected components as a library step);
  * the sample chooser, written from its definition (bottom-k of splitmix64
    keys);
  * ctypes calls into cc_oracle.c for BFS / Dijkstra, the k x n distance
    table and the estimators of section 2 (eqs. (1), (3), (4));
  * node-weighted closeness (section 5) in plain Python integers: the
    threshold tau, the exact-size weighted sample and the sampling and
    hybrid estimates of S_beta from a distance table;
  * outbound / inbound estimates of general directed graphs (section 6.2):
    per node the bottom-k sample of its reachability set by rank, from an
    all-pairs table.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libcc_oracle.so")
_lib = None

INF = 0xFFFFFFFF
EST_NAMES = ("sampling", "pivoting", "pivot_upper", "hybrid")


def build(force: bool = False) -> str:
    """Compile cc_oracle.c into oracle/_build/libcc_oracle.so with gcc."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or (
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        i64, i32, u32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32
        lib.orc_bfs.argtypes = [i64, P, P, i32, P]
        lib.orc_dijkstra.argtypes = [i64, P, P, P, i32, P]
        lib.orc_dist_table.argtypes = [i64, P, P, P, i32, P, P]
        lib.orc_roundtrip_table.argtypes = [i64, P, P, P, P, P, P, i32, P, P]
        lib.orc_exact_S.argtypes = [i64, P, P, P, P]
        lib.orc_estimate.argtypes = [i64, i32, P, P, u32, u32, P, P, P, P, P,
                                     P, P, P]
        lib.orc_closeness_from_S.argtypes = [i64, P, P]
        lib.orc_streaming_pass.argtypes = [i64, P, P, P, i32, P, P, P, P, P]
        lib.orc_sqerr.argtypes = [i64, i32, P, P, u32, u32, P, P]
        lib.orc_adaptive.argtypes = [i64, i32, P, P, i32, P, P, P, P, P]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


# --------------------------------------------------------------------------
# Graph building
# --------------------------------------------------------------------------

class Graph:
    """A CSR graph as the oracle builds it.

    row_ptr int64[n+1], col int32[row_ptr[n]], w uint32 or None, old_id int32[n]
    (original id of each kept node).  Directed graphs also carry the CSR of
    the reversed graph (rrow_ptr, rcol, rw).
    """

    def __init__(self, n, row_ptr, col, w, old_id, directed,
                 rrow_ptr=None, rcol=None, rw=None):
        self.n = int(n)
        self.row_ptr = row_ptr
        self.col = col
        self.w = w
        self.old_id = old_id
        self.directed = directed
        self.rrow_ptr, self.rcol, self.rw = rrow_ptr, rcol, rw

    @property
    def arcs(self):
        return int(self.row_ptr[-1])

    @property
    def m(self):
        """Undirected edges (each counted once) or directed arcs."""
        return self.arcs if self.directed else self.arcs // 2


def _dedup_arcs(n, s, d, w):
    """Sort arcs by (s, d) and keep one per pair (the smallest weight)."""
    key = s.astype(np.int64) * n + d.astype(np.int64)
    if w is None:
        key = np.sort(key)
        first = np.ones(key.size, dtype=bool)
        first[1:] = key[1:] != key[:-1]
        key = key[first]
        return (key // n).astype(np.int64), (key % n).astype(np.int64), None
    order = np.lexsort((w, key))
    key, w = key[order], w[order]
    first = np.ones(key.size, dtype=bool)
    first[1:] = key[1:] != key[:-1]
    key, w = key[first], w[first]
    return (key // n).astype(np.int64), (key % n).astype(np.int64), w


def _csr(n, s, d, w):
    counts = np.bincount(s, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, d.astype(np.int32), (None if w is None else w.astype(np.uint32))


def _largest(labels):
    """Label of the largest component; ties go to the component holding the
    smallest node id."""
    sizes = np.bincount(labels)
    best = sizes.max()
    cands = np.flatnonzero(sizes == best)
    if cands.size == 1:
        return int(cands[0])
    first_node = np.full(labels.max() + 1, np.iinfo(np.int64).max)
    np.minimum.at(first_node, labels, np.arange(labels.size))
    return int(cands[np.argmin(first_node[cands])])


def csr_from_edges(n, src, dst, w=None, directed=False, keep_component=True):
    """Build the graph the estimators run on (step "graph to CSR").

    Undirected: every edge gives arcs both ways.  Self-loops are dropped and
    parallel arcs merged (keeping the smallest weight).  With keep_component,
    only the largest connected component (strongly connected for directed
    input) is kept, its nodes renumbered 0..n'-1 in increasing original id.
    Adjacency lists are sorted by neighbour id.
    """
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components

    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    ww = None if w is None else np.asarray(w, dtype=np.uint32)
    if directed:
        s, d = src, dst
    else:
        s, d = np.concatenate([src, dst]), np.concatenate([dst, src])
        if ww is not None:
            ww = np.concatenate([ww, ww])
    keep = s != d
    s, d = s[keep], d[keep]
    if ww is not None:
        ww = ww[keep]
    s, d, ww = _dedup_arcs(n, s, d, ww)

    old_id = np.arange(n, dtype=np.int64)
    if keep_component:
        adj = csr_matrix((np.ones(s.size, dtype=np.int8), (s, d)), shape=(n, n))
        _, labels = connected_components(
            adj, directed=directed, connection="strong" if directed else "weak")
        lab = _largest(labels)
        kept = labels == lab
        old_id = np.flatnonzero(kept)
        new_id = np.full(n, -1, dtype=np.int64)
        new_id[old_id] = np.arange(old_id.size)
        arc_ok = kept[s] & kept[d]
        s, d = new_id[s[arc_ok]], new_id[d[arc_ok]]
        if ww is not None:
            ww = ww[arc_ok]
        n = old_id.size
    row_ptr, col, wout = _csr(n, s, d, ww)
    g = Graph(n, row_ptr, col, wout, old_id.astype(np.int32), directed)
    if directed:
        order = np.lexsort((s, d))
        g.rrow_ptr, g.rcol, g.rw = _csr(n, d[order], s[order],
                                        None if ww is None else ww[order])
    return g


# --------------------------------------------------------------------------
# Sample chooser: bottom-k of splitmix64 keys
# --------------------------------------------------------------------------

_G = 0x9E3779B97F4A7C15
_MASK = (1 << 64) - 1


def splitmix64_key(seed: int, v: int) -> int:
    """Pure-integer splitmix64 output number v of stream `seed` (Steele, Lea
    and Flood 2014): mix(seed + (v+1)*gamma)."""
    z = (seed + (v + 1) * _G) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def choose_sample(n: int, k: int, seed: int) -> np.ndarray:
    """Uniform sample of k distinct nodes (section 2: "sample k points
    uniformly at random"): node v gets the key splitmix64_key(seed, v) and
    the sample is the k nodes with the smallest (key, v), in that order --
    a bottom-k sample, uniform without replacement.  The order fixes each
    node's sample index."""
    if not (0 < k <= n):
        raise ValueError("need 0 < k <= n")
    keys = np.array([splitmix64_key(seed, v) for v in range(n)], dtype=np.uint64) \
        if n <= 4096 else _keys_vec(seed, n)
    order = np.lexsort((np.arange(n), keys))
    return order[:k].astype(np.int32)


def _keys_vec(seed, n):
    c = np.arange(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + (c + np.uint64(1)) * np.uint64(_G)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


# --------------------------------------------------------------------------
# Distances and estimators
# --------------------------------------------------------------------------

def bfs(g: Graph, s: int, reverse=False) -> np.ndarray:
    rp, col = (g.rrow_ptr, g.rcol) if reverse else (g.row_ptr, g.col)
    dist = np.empty(g.n, dtype=np.uint32)
    _check(_L().orc_bfs(g.n, _p(rp), _p(col), int(s), _p(dist)), "bfs")
    return dist


def sssp(g: Graph, s: int, reverse=False) -> np.ndarray:
    """Distances from s: BFS when unweighted, Dijkstra otherwise."""
    rp, col, w = ((g.rrow_ptr, g.rcol, g.rw) if reverse
                  else (g.row_ptr, g.col, g.w))
    dist = np.empty(g.n, dtype=np.uint32)
    if w is None:
        rc = _L().orc_bfs(g.n, _p(rp), _p(col), int(s), _p(dist))
    else:
        rc = _L().orc_dijkstra(g.n, _p(rp), _p(col), _p(w), int(s), _p(dist))
    _check(rc, "sssp")
    return dist


def dist_table(g: Graph, sources, roundtrip=False) -> np.ndarray:
    """k x n table of d(c_i, v) (round-trip d(c_i,v)+d(v,c_i) if asked)."""
    src = np.ascontiguousarray(sources, dtype=np.int32)
    k = src.size
    table = np.empty((k, g.n), dtype=np.uint32)
    if roundtrip:
        rc = _L().orc_roundtrip_table(g.n, _p(g.row_ptr), _p(g.col), _p(g.w),
                                      _p(g.rrow_ptr), _p(g.rcol), _p(g.rw),
                                      k, _p(src), _p(table))
    else:
        rc = _L().orc_dist_table(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), k,
                                 _p(src), _p(table))
    _check(rc, "dist_table")
    return table


def exact_S(g: Graph, roundtrip=False) -> np.ndarray:
    """S(v) = sum_u d(v,u) by n SSSPs (eq. (1)); round-trip adds the
    reversed graph's sums."""
    S = np.empty(g.n, dtype=np.uint64)
    _check(_L().orc_exact_S(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), _p(S)),
           "exact_S")
    if roundtrip:
        R = np.empty(g.n, dtype=np.uint64)
        _check(_L().orc_exact_S(g.n, _p(g.rrow_ptr), _p(g.rcol), _p(g.rw),
                                _p(R)), "exact_S")
        S = S + R
    return S


def exact_closeness(S: np.ndarray) -> np.ndarray:
    out = np.empty(S.size, dtype=np.float64)
    _check(_L().orc_closeness_from_S(S.size, _p(np.ascontiguousarray(S)),
                                     _p(out)), "closeness")
    return out


def estimate_from_table(table: np.ndarray, sources, eps=(1, 8)):
    """Every statistic and estimate of section 2 from a k x n metric table.

    Returns a dict with pivot, delta, sum, S_samp, delta_cc (k x k),
    hyb (n x 6: Hsum, Hnum, HCsum, LCsum, LCnum, LCsumSq), s_hat (4 x n),
    closeness (4 x n), rows in the order sampling, pivoting, pivot_upper,
    hybrid.
    """
    table = np.ascontiguousarray(table, dtype=np.uint32)
    k, n = table.shape
    src = np.ascontiguousarray(sources, dtype=np.int32)
    out = dict(
        pivot=np.empty(n, np.int32), delta=np.empty(n, np.uint32),
        sum=np.empty(n, np.uint64), S_samp=np.empty(k, np.uint64),
        delta_cc=np.empty((k, k), np.uint32), hyb=np.empty((n, 6), np.uint64),
        s_hat=np.empty((4, n), np.float64),
        closeness=np.empty((4, n), np.float64))
    rc = _L().orc_estimate(n, k, _p(src), _p(table), int(eps[0]), int(eps[1]),
                           _p(out["pivot"]), _p(out["delta"]), _p(out["sum"]),
                           _p(out["S_samp"]), _p(out["delta_cc"]),
                           _p(out["hyb"]), _p(out["s_hat"]),
                           _p(out["closeness"]))
    _check(rc, "estimate")
    return out


def pass1_from_table(table: np.ndarray, sources):
    """The first-pass statistics of estimate_from_table alone -- pivot,
    delta, sum, S_samp, delta_cc -- without its estimates (whose H tail
    costs O(n) per node)."""
    table = np.ascontiguousarray(table, dtype=np.uint32)
    k, n = table.shape
    src = np.ascontiguousarray(sources, dtype=np.int32)
    out = dict(pivot=np.empty(n, np.int32), delta=np.empty(n, np.uint32),
               sum=np.empty(n, np.uint64), S_samp=np.empty(k, np.uint64),
               delta_cc=np.empty((k, k), np.uint32))
    rc = _L().orc_estimate(n, k, _p(src), _p(table), 1, 1, _p(out["pivot"]),
                           _p(out["delta"]), _p(out["sum"]), _p(out["S_samp"]),
                           _p(out["delta_cc"]), None, None, None)
    _check(rc, "pass1")
    return out


def estimate(g: Graph, sources, eps=(1, 8), roundtrip=False):
    """dist_table + estimate_from_table."""
    return estimate_from_table(dist_table(g, sources, roundtrip), sources, eps)


# The eps values of the adaptive hybrid (section 6): 0.001, 0.025, 0.05,
# 0.1, 0.2, 0.5 and 0.99, as fractions a/b.
ADAPTIVE_EPS = ((1, 1000), (1, 40), (1, 20), (1, 10), (1, 5), (1, 2), (99, 100))


def sqerr_from_table(table: np.ndarray, sources, eps=(1, 8)):
    """Hybrid estimate of S and its error estimate SqErrEst (Algorithm 1's
    last loop; section 4) for every node, from a k x n metric table.
    Returns (s_hat, sqerr); sampled nodes get their exact S and error 0."""
    table = np.ascontiguousarray(table, dtype=np.uint32)
    k, n = table.shape
    src = np.ascontiguousarray(sources, dtype=np.int32)
    s_hat = np.empty(n, np.float64)
    sqerr = np.empty(n, np.float64)
    rc = _L().orc_sqerr(n, k, _p(src), _p(table), int(eps[0]), int(eps[1]), _p(s_hat),
                        _p(sqerr))
    _check(rc, "sqerr")
    return s_hat, sqerr


def adaptive_from_table(table: np.ndarray, sources, eps_list=ADAPTIVE_EPS):
    """The adaptive hybrid (section 6): per node the hybrid estimate under
    the eps of eps_list with the smallest SqErrEst.  Returns (s_hat, sqerr,
    choice) with choice = position in eps_list (-1 for sampled nodes)."""
    table = np.ascontiguousarray(table, dtype=np.uint32)
    k, n = table.shape
    src = np.ascontiguousarray(sources, dtype=np.int32)
    a = np.ascontiguousarray([e[0] for e in eps_list], dtype=np.uint32)
    b = np.ascontiguousarray([e[1] for e in eps_list], dtype=np.uint32)
    s_hat = np.empty(n, np.float64)
    sqerr = np.empty(n, np.float64)
    choice = np.empty(n, np.int32)
    rc = _L().orc_adaptive(n, k, _p(src), _p(table), len(eps_list), _p(a), _p(b), _p(s_hat),
                           _p(sqerr), _p(choice))
    _check(rc, "adaptive")
    return s_hat, sqerr, choice


def streaming_pass(g: Graph, sources):
    """k SSSPs with O(1) running state per node (section 3): sum, pivot,
    Delta and the exact S of each sampled node.  Timed for the CPU
    baseline; equal to the table-based statistics."""
    src = np.ascontiguousarray(sources, dtype=np.int32)
    k = src.size
    s = np.empty(g.n, np.uint64)
    piv = np.empty(g.n, np.int32)
    dl = np.empty(g.n, np.uint32)
    S = np.empty(k, np.uint64)
    _check(_L().orc_streaming_pass(g.n, _p(g.row_ptr), _p(g.col), _p(g.w), k,
                                   _p(src), _p(s), _p(piv), _p(dl), _p(S)),
           "streaming_pass")
    return dict(sum=s, pivot=piv, delta=dl, S_samp=S)


def default_eps(k: int):
    """eps = 1/sqrt(k) as the rational 1/round(sqrt(k)) (section 7 uses
    eps = sqrt(1/k); the garbled "eps = sqrt k" of section 2 is read so)."""
    return (1, max(1, int(round(k ** 0.5))))


# --------------------------------------------------------------------------
# Node-weighted closeness (section 5, "Weighted Centrality")
# --------------------------------------------------------------------------
#
# Node weights beta(v) >= 0 (integers here).  S_beta(v) = sum over u != v of
# beta(u) d(v, u) and the closeness is (sum of beta - beta(v)) / S_beta(v)
# (eq. (2) read with the weight of the other endpoint j, as the text after it
# computes the numerator).  The sample has exactly k nodes; node v is in it
# with probability min(1, beta(v) / tau) and counts with the adjusted weight
# max(tau, beta(v)).  tau is kept as the exact rational tn / td.


def varopt_threshold(beta, k: int):
    """The threshold tau = tn / td of section 5: the value with
    sum over v of min(1, beta(v) / tau) = k.  With the weights sorted
    b_0 >= b_1 >= ..., the h largest are taken with certainty and the rest in
    proportion to weight, tau = (b_h + b_{h+1} + ...) / (k - h), for the
    smallest h at which b_h < tau (then b_{h-1} >= tau holds too).  When
    exactly k weights are positive every one of them is certain and
    tau = (smallest positive weight) / 1."""
    b = sorted((int(x) for x in beta if int(x) > 0), reverse=True)
    if not 0 < k <= len(b):
        raise ValueError("need 0 < k <= number of positive weights")
    if len(b) == k:
        return b[-1], 1
    rest = sum(b)                      # b_h + b_{h+1} + ..., for h = 0
    for h in range(k):
        if b[h] * (k - h) < rest:      # b_h < rest / (k - h)
            return rest, k - h
        rest -= b[h]
    raise AssertionError("unreachable: more than k positive weights")


def is_certain(b: int, tau) -> bool:
    """beta >= tau (inclusion probability 1), for a positive weight."""
    return b * tau[1] >= tau[0]


def systematic_pick(order, beta, tau, u: int):
    """Systematic sampling with unequal probabilities (Madow 1949) of the
    uncertain nodes along `order`: node v occupies the interval of length
    beta(v) * td in a line of total length td * tn, and the td points
    u, u + tn, u + 2 tn, ... (0 <= u < tn) pick the nodes whose interval
    holds one; an interval shorter than tn holds at most one point, so node v
    is picked for exactly beta(v) * td of the tn offsets u -- probability
    beta(v) / tau.  Certain nodes are always picked, zero weights never.
    Returns the picked nodes in `order`."""
    tn, td = tau
    picked = []
    pos = 0

    def points_below(x):               # points u + t tn (t >= 0) below x
        return 0 if x <= u else (x - u + tn - 1) // tn

    for v in order:
        b = int(beta[v])
        if b == 0:
            continue
        if is_certain(b, tau):
            picked.append(int(v))
            continue
        lo, pos = pos, pos + b * td
        if points_below(pos) > points_below(lo):
            picked.append(int(v))
    return picked


def sample_order(n: int, seed: int) -> np.ndarray:
    """Nodes in increasing (splitmix64_key(seed, v), v): a uniformly random
    order, the same keys as choose_sample."""
    keys = np.array([splitmix64_key(seed, v) for v in range(n)], dtype=np.uint64) \
        if n <= 4096 else _keys_vec(seed, n)
    return np.lexsort((np.arange(n), keys))


def sample_varopt(beta, k: int, seed: int):
    """Weighted sample of exactly k nodes (section 5): inclusion probability
    min(1, beta(v) / tau) by systematic sampling along a random order; the
    offset u is splitmix64 output number n of the stream `seed` scaled to
    [0, tn) by a 64 x 64 -> 128-bit product (its high half).  Returns
    (sample as int32 in the order's sequence, (tn, td))."""
    beta = np.asarray(beta)
    n = beta.size
    tau = varopt_threshold(beta, k)
    u = (splitmix64_key(seed, n) * tau[0]) >> 64
    C = systematic_pick(sample_order(n, seed), beta, tau, u)
    assert len(C) == k
    return np.asarray(C, dtype=np.int32), tau


def node_weighted_from_table(table: np.ndarray, sources, beta, tau, eps=(1, 8)):
    """Node-weighted estimates of S_beta from a k x n metric table (section
    5 and its modification of Algorithm 1).

    Sampled node c_i: exact S_beta(c_i) = sum_u beta(u) d(c_i, u).
    Other node v, with pivot p = c(v) (nearest sampled node, smallest index
    on ties) and Delta = d(p, v); x is "beyond" when x a > Delta b (eps =
    a/b):
      sampling (inverse-probability) estimate:
          sum over c in C of max(tau, beta(c)) d(c, v);
      hybrid: every non-sampled w beyond from p counts beta(w) d(p, w)
          (the H tail), every sampled c_i with d(p, c_i) beyond counts
          beta(c_i) d(c_i, v) (HC), and the other sampled nodes count
          max(tau, beta(c_i)) d(c_i, v) (the estimate of L).
    Returns dict(S_samp (k, exact integers), num (2 x n numerators over td,
    Python ints; sampled nodes hold S * td), s_hat (2 x n), closeness
    (2 x n)), rows in the order sampling, hybrid."""
    T = np.asarray(table, dtype=np.int64)
    k, n = T.shape
    C = [int(c) for c in sources]
    beta = [int(x) for x in beta]
    tn, td = int(tau[0]), int(tau[1])
    a, b = int(eps[0]), int(eps[1])
    bC = np.array([beta[c] for c in C], dtype=np.int64)
    certain = np.array([is_certain(x, (tn, td)) for x in bC.tolist()], dtype=bool)
    bvec = np.array(beta, dtype=np.int64)
    S_samp = [int((bvec * T[i]).sum()) for i in range(k)]
    sidx = {c: i for i, c in enumerate(C)}
    notC = np.ones(n, dtype=bool)
    notC[C] = False
    total = sum(beta)
    num = [[0] * n, [0] * n]
    for v in range(n):
        if v in sidx:
            num[0][v] = num[1][v] = S_samp[sidx[v]] * td
            continue
        col = T[:, v]
        # tau * sum of d over uncertain samples + beta * d over certain ones
        num[0][v] = (tn * int(col[~certain].sum()) +
                     td * int((bC[certain] * col[certain]).sum()))
        p = int(np.argmin(col))          # first minimum: smallest index
        delta = int(col[p])
        row = T[p]
        H = notC & (row * a > delta * b)
        Hsum = int((bvec[H] * row[H]).sum())
        HC = row[C] * a > delta * b
        HCsum = int((bC[HC] * col[HC]).sum())
        LC = ~HC
        Lpart = (tn * int(col[LC & ~certain].sum()) +
                 td * int((bC[LC & certain] * col[LC & certain]).sum()))
        num[1][v] = td * (Hsum + HCsum) + Lpart
    from fractions import Fraction
    s_hat = np.array([[float(Fraction(x, td)) for x in row] for row in num])
    wsum = np.array([float(total - beta[v]) for v in range(n)])
    with np.errstate(divide="ignore", invalid="ignore"):
        clo = wsum[None, :] / s_hat
    return dict(S_samp=S_samp, num=num, s_hat=s_hat, closeness=clo)


def exact_weighted_S(table_all: np.ndarray, beta):
    """S_beta(v) = sum_u beta(u) d(v, u) from an n x n table (rows: v)."""
    T = np.asarray(table_all, dtype=np.int64)
    bvec = np.asarray([int(x) for x in beta], dtype=np.int64)
    return [int((T[v] * bvec).sum()) for v in range(T.shape[0])]


# --------------------------------------------------------------------------
# Outbound / inbound estimates for general directed graphs (section 6.2,
# Algorithm 4)
# --------------------------------------------------------------------------
#
# For node v, R(v) = the nodes u != v that v reaches (outbound; inbound: that
# reach v) and S(v) = the sum of d(v, u) over them.  With the nodes in one
# random order (rank), v's sample is the k nodes of R(v) of smallest rank;
# the estimates are the average distance to the sample and a bottom-k
# estimate of |R(v)| from the rank position of the k-th sample.


def reach_from_table(table_all: np.ndarray, order, k: int, inbound=False):
    """Per node, from the n x n distance table (row u: d(u, .); unreachable
    = INF): count = min(k, |R(v)|), distsum = sum of the distances to the
    sample, T = the position (1-based, among the nodes other than v) of the
    k-th sample in the order, 0 when count < k; avg = distsum / count (0
    when count = 0), R_hat = count when count < k, else
    1 + (k - 1)(n - 2) / (T - 1).  Returns a dict of arrays."""
    D = np.asarray(table_all, dtype=np.int64)
    n = D.shape[0]
    order = [int(x) for x in order]
    pos = {u: p for p, u in enumerate(order)}          # 0-based rank position
    count = np.zeros(n, np.int32)
    distsum = np.zeros(n, np.uint64)
    T = np.zeros(n, np.int64)
    avg = np.zeros(n)
    R_hat = np.zeros(n)
    for v in range(n):
        dist = D[:, v] if inbound else D[v, :]
        reach = [u for u in order if u != v and dist[u] != INF]   # rank order
        sample = reach[:k]
        count[v] = len(sample)
        distsum[v] = sum(int(dist[u]) for u in sample)
        if count[v]:
            avg[v] = int(distsum[v]) / int(count[v])
        if count[v] < k:
            R_hat[v] = count[v]
        else:
            t = pos[sample[-1]] + 1                         # 1-based position
            T[v] = t - 1 if pos[v] < pos[sample[-1]] else t  # not counting v
            # k = 1: the numerator (k - 1)(n - 2) is 0 and R_hat = 1
            R_hat[v] = 1.0 if k == 1 else 1.0 + float((k - 1) * (n - 2)) / float(T[v] - 1)
    return dict(count=count, distsum=distsum, T=T, avg=avg, R_hat=R_hat)


def all_pairs(g: Graph) -> np.ndarray:
    """n x n table of d(u, v) (row u), INF where v is unreachable: one BFS
    (Dijkstra with arc lengths) per node."""
    return np.stack([sssp(g, u) for u in range(g.n)])


# --------------------------------------------------------------------------
# One node at a time (undirected graphs of any size)
# --------------------------------------------------------------------------

def _metric_from(g: Graph, x: int, roundtrip: bool) -> np.ndarray:
    """d(x, .) (undirected), or the round-trip d(x, .) + d(., x) (section
    6.1: a search on G plus one on G^T)."""
    d = sssp(g, x).astype(np.int64)
    if roundtrip:
        back = sssp(g, x, reverse=True).astype(np.int64)
        d = np.where((d == INF) | (back == INF), INF, d + back)
    return d


def estimate_node(g: Graph, sources, v: int, eps=(1, 8), roundtrip=False):
    """Every statistic and estimate of section 2 for the single node v, from
    searches out of v (its distance to every sampled node, and S(v)) and out
    of its pivot p (the H tail d(p, w) over V \\ C, delta(p, c_i) and S(p)):
    one search each on an undirected graph, a forward and a reversed one
    each for round trips (section 6.1).  Same definitions as
    estimate_from_table: pivot = the nearest sampled node, smallest index on
    ties; x beyond when x a > Delta b; eq. (4) with the numerator
    (Hsum + HCsum) |L n C| + LCsum |L| formed exactly and divided once.
    Returns dict(pivot, delta, sum, s_hat (4 floats), hyb (the six
    integers Hsum, Hnum, HCsum, LCsum, LCnum, LCsumSq; zeros for v in C))."""
    assert roundtrip == g.directed
    C = [int(c) for c in sources]
    k, n = len(C), g.n
    a, b = int(eps[0]), int(eps[1])
    dv = _metric_from(g, v, roundtrip)
    dC = np.array([dv[c] for c in C], dtype=np.int64)      # d(c_i, v)
    sidx = {c: i for i, c in enumerate(C)}
    total = int(dC.sum())
    if v in sidx:
        Sv = int(dv.sum())
        return dict(pivot=sidx[v], delta=0, sum=total, s_hat=[float(Sv)] * 4,
                    hyb=[0] * 6)
    i_p = int(np.argmin(dC))                                # first minimum
    delta = int(dC[i_p])
    dp = _metric_from(g, C[i_p], roundtrip)
    Sp = int(dp.sum())
    from fractions import Fraction
    s_samp = float(Fraction((n - 1) * total, k))
    s_piv = float(Sp)
    s_up = float(Sp + (n - 1) * delta)
    notC = np.ones(n, dtype=bool)
    notC[C] = False
    H = notC & (dp * a > delta * b)
    Hsum, Hnum = int(dp[H].sum()), int(H.sum())
    HC = np.array([dp[c] * a > delta * b for c in C])
    HCsum = int(dC[HC].sum())
    LCnum = int((~HC).sum())
    LCsum = int(dC[~HC].sum())
    LCsumSq = sum(int(x) * int(x) for x in dC[~HC])
    Lnum = (n - 1) - Hnum - int(HC.sum())
    s_hyb = float(Fraction((Hsum + HCsum) * LCnum + LCsum * Lnum, LCnum))
    return dict(pivot=i_p, delta=delta, sum=total, s_hat=[s_samp, s_piv, s_up, s_hyb],
                hyb=[Hsum, Hnum, HCsum, LCsum, LCnum, LCsumSq])


def reach_node(g: Graph, order, v: int, k: int, inbound=False):
    """reach_from_table for the single node v, from one search out of v
    (on G for outbound, on G^T for inbound).  Returns dict(count, distsum,
    T, avg, R_hat) for v."""
    n = g.n
    dist = sssp(g, v, reverse=inbound).astype(np.int64)
    order = np.asarray(order, dtype=np.int64)
    pos = np.empty(n, dtype=np.int64)
    pos[order] = np.arange(n)
    reach = order[(dist[order] != INF) & (order != v)]   # in rank order
    sample = reach[:k]
    count = int(sample.size)
    distsum = int(dist[sample].sum())
    T, R_hat = 0, float(count)
    if count == k:
        t = int(pos[sample[-1]]) + 1
        T = t - 1 if pos[v] < pos[sample[-1]] else t
        R_hat = 1.0 if k == 1 else 1.0 + float((k - 1) * (n - 2)) / float(T - 1)
    return dict(count=count, distsum=distsum, T=T,
                avg=(distsum / count if count else 0.0), R_hat=R_hat)


def node_weighted_node(g: Graph, sources, beta, tau, v: int, eps=(1, 8), roundtrip=False):
    """node_weighted_from_table for the single node v, from searches out of
    v and out of its pivot (as estimate_node).  Returns dict(num (2 Python
    ints over td), s_hat (2 floats), closeness (2 floats))."""
    from fractions import Fraction
    C = [int(c) for c in sources]
    beta = [int(x) for x in beta]
    tn, td = int(tau[0]), int(tau[1])
    a, b = int(eps[0]), int(eps[1])
    n = g.n
    bvec = np.asarray(beta, dtype=np.int64)
    total = int(bvec.sum())
    dv = _metric_from(g, v, roundtrip)
    sidx = {c: i for i, c in enumerate(C)}
    if v in sidx:
        S = int((bvec * dv).sum())
        num = [S * td, S * td]
    else:
        col = np.array([dv[c] for c in C], dtype=np.int64)
        bC = np.array([beta[c] for c in C], dtype=np.int64)
        certain = np.array([is_certain(x, (tn, td)) for x in bC.tolist()], dtype=bool)
        num0 = tn * int(col[~certain].sum()) + td * int((bC[certain] * col[certain]).sum())
        i_p = int(np.argmin(col))
        delta = int(col[i_p])
        row = _metric_from(g, C[i_p], roundtrip)
        notC = np.ones(n, dtype=bool)
        notC[C] = False
        H = notC & (row * a > delta * b)
        Hsum = int((bvec[H] * row[H]).sum())
        HC = np.array([row[c] * a > delta * b for c in C])
        HCsum = int((bC[HC] * col[HC]).sum())
        LC = ~HC
        Lpart = (tn * int(col[LC & ~certain].sum()) +
                 td * int((bC[LC & certain] * col[LC & certain]).sum()))
        num = [num0, td * (Hsum + HCsum) + Lpart]
    s_hat = [float(Fraction(x, td)) for x in num]
    wv = float(total - beta[v])
    return dict(num=num, s_hat=s_hat, closeness=[wv / x if x else float("nan") for x in s_hat])
