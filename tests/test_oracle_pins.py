"""Pins for the CPU oracle: closed forms, hand-derived examples, published
test vectors, brute force by a different algorithm and invariants of the
method.  CPU only."""
import collections
import heapq
import itertools
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import oracle as orc
from tests.golden import load as golden


def G(gen, *args, w=None, directed=False, keep=True):
    n, s, d = gen(*args)
    return orc.csr_from_edges(n, s, d, w=w, directed=directed,
                              keep_component=keep)


# ---------------------------------------------------------------- distances

def f_line(p, n):
    """Sum of distances from position p on a path of n nodes."""
    return p * (p + 1) // 2 + (n - 1 - p) * (n - p) // 2


@pytest.mark.parametrize("n", [2, 3, 7, 30])
def test_bfs_path_cycle_closed_forms(n):
    g = G(synth.path_edges, n)
    for s in range(n):
        assert (orc.bfs(g, s) == np.abs(np.arange(n) - s)).all()
    if n >= 3:
        c = G(synth.cycle_edges, n)
        for s in range(n):
            d = np.abs(np.arange(n) - s)
            assert (orc.bfs(c, s) == np.minimum(d, n - d)).all()


def test_bfs_grid_is_manhattan():
    a, b = 7, 5
    g = G(synth.grid_edges, a, b)
    xs, ys = np.arange(a * b) % a, np.arange(a * b) // a
    for s in [0, 3, 17, a * b - 1]:
        want = np.abs(xs - xs[s]) + np.abs(ys - ys[s])
        assert (orc.bfs(g, s) == want).all()


def floyd_warshall(n, row_ptr, col, w):
    D = np.full((n, n), np.iinfo(np.int64).max // 4, dtype=np.int64)
    np.fill_diagonal(D, 0)
    for u in range(n):
        for e in range(row_ptr[u], row_ptr[u + 1]):
            v = col[e]
            D[u, v] = min(D[u, v], 1 if w is None else int(w[e]))
    for m in range(n):
        D = np.minimum(D, D[:, m:m + 1] + D[m:m + 1, :])
    return D


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_dijkstra_matches_floyd_warshall(seed):
    n, s, d = synth.watts_strogatz_edges(40, 4, 0.3, seed=seed)
    w = synth.random_weights(s.size, 1, 50, seed=seed + 10)
    g = orc.csr_from_edges(n, s, d, w=w)
    D = floyd_warshall(g.n, g.row_ptr, g.col, g.w)
    for src in range(g.n):
        assert (orc.sssp(g, src).astype(np.int64) == D[src]).all()
    Du = floyd_warshall(g.n, g.row_ptr, g.col, None)
    for src in range(g.n):
        assert (orc.bfs(g, src).astype(np.int64) == Du[src]).all()


def test_dijkstra_directed_matches_floyd_warshall():
    n, s, d = synth.rmat_edges(6, 6, seed=5)
    w = synth.random_weights(s.size, 1, 9, seed=6)
    g = orc.csr_from_edges(n, s, d, w=w, directed=True)
    D = floyd_warshall(g.n, g.row_ptr, g.col, g.w)
    R = floyd_warshall(g.n, g.rrow_ptr, g.rcol, g.rw)
    assert (D == R.T).all()  # reversed graph = transposed distances
    for src in range(0, g.n, 3):
        assert (orc.sssp(g, src).astype(np.int64) == D[src]).all()
        assert (orc.sssp(g, src, reverse=True).astype(np.int64) == D[:, src]).all()


# ---------------------------------------------------------------- exact S

def test_exact_S_closed_forms():
    n = 12
    assert list(orc.exact_S(G(synth.path_edges, n))) == [f_line(p, n) for p in range(n)]
    S = orc.exact_S(G(synth.star_edges, n))
    assert S[0] == n - 1 and (S[1:] == 2 * n - 3).all()
    for n in (5, 8):
        assert (orc.exact_S(G(synth.cycle_edges, n)) == n * n // 4).all()
    assert (orc.exact_S(G(synth.complete_edges, 9)) == 8).all()
    a, b = 6, 4
    S = orc.exact_S(G(synth.grid_edges, a, b))
    for v in range(a * b):
        x, y = v % a, v // a
        assert S[v] == b * f_line(x, a) + a * f_line(y, b)
    cl = orc.exact_closeness(orc.exact_S(G(synth.path_edges, 5)))
    assert cl[2] == 4 / 6  # eq. (1): (n-1) / sum of distances


def test_roundtrip_closed_forms():
    # directed cycle: d(u,v) + d(v,u) = n for u != v -> S = n(n-1)
    n = 9
    s = np.arange(n, dtype=np.uint32)
    g = orc.csr_from_edges(n, s, (s + 1) % n, directed=True)
    assert (orc.exact_S(g, roundtrip=True) == n * (n - 1)).all()
    tab = orc.dist_table(g, [0, 4], roundtrip=True)
    assert (tab == np.where(np.arange(n) == np.array([[0], [4]]), 0, n)).all()
    # both orientations of an undirected path: round trip = twice the distance
    m, a, b = synth.path_edges(6)
    gd = orc.csr_from_edges(m, np.concatenate([a, b]), np.concatenate([b, a]),
                            directed=True)
    assert list(orc.exact_S(gd, roundtrip=True)) == [2 * f_line(p, 6) for p in range(6)]


# ---------------------------------------------------------------- sampler

def test_splitmix64_published_vectors():
    for row in golden.read("splitmix64.txt")["seed"]:
        seed = int(row[0])
        for c, hx in enumerate(row[1:]):
            assert orc.splitmix64_key(seed, c) == int(hx, 16)
            assert int(synth.splitmix64_at(seed, [c])[0]) == int(hx, 16)


def test_sample_is_bottom_k_and_uniform():
    n, k = 10, 3
    for seed in range(5):
        c = orc.choose_sample(n, k, seed)
        keys = [orc.splitmix64_key(seed, v) for v in range(n)]
        want = sorted(range(n), key=lambda v: (keys[v], v))[:k]
        assert list(c) == want and len(set(c)) == k
    assert (orc.choose_sample(5000, 40, 7) == orc.choose_sample(5000, 40, 7)).all()
    # inclusion frequency ~ k/n (statistical, loose)
    counts = np.zeros(n)
    for seed in range(4000):
        counts[orc.choose_sample(n, k, seed)] += 1
    assert np.abs(counts / 4000 - k / n).max() < 0.04
    with pytest.raises(ValueError):
        orc.choose_sample(4, 5, 0)


# ---------------------------------------------------------------- graph build

def brute_graph(n, src, dst, w, directed):
    arcs = {}
    for i, (u, v) in enumerate(zip(src.tolist(), dst.tolist())):
        if u == v:
            continue
        ww = 1 if w is None else int(w[i])
        pairs = [(u, v)] if directed else [(u, v), (v, u)]
        for p in pairs:
            arcs[p] = min(arcs.get(p, ww), ww)
    reach = np.eye(n, dtype=bool)
    for (u, v) in arcs:
        reach[u, v] = True
    for m in range(n):
        reach |= reach[:, m:m + 1] & reach[m:m + 1, :]
    comp = reach & reach.T
    labels = [min(np.flatnonzero(comp[v])) for v in range(n)]
    sizes = collections.Counter(labels)
    best = max(sizes.values())
    lab = min(l for l, s in sizes.items() if s == best)  # holds smallest id
    keep = [v for v in range(n) if labels[v] == lab]
    new = {v: i for i, v in enumerate(keep)}
    rows = [[] for _ in keep]
    for (u, v), ww in arcs.items():
        if u in new and v in new:
            rows[new[u]].append((new[v], ww))
    return keep, [sorted(r) for r in rows]


@pytest.mark.parametrize("directed", [False, True])
@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_csr_build_matches_brute_force(directed, seed):
    n = 24
    rng = np.random.default_rng(seed)
    m = 40
    src = rng.integers(0, n, m).astype(np.uint32)
    dst = rng.integers(0, n, m).astype(np.uint32)
    src[:3] = dst[:3]  # self-loops
    src, dst = np.concatenate([src, src[:5]]), np.concatenate([dst, dst[:5]])
    w = rng.integers(1, 9, src.size).astype(np.uint32)
    g = orc.csr_from_edges(n, src, dst, w=w, directed=directed)
    keep, rows = brute_graph(n, src, dst, w, directed)
    assert list(g.old_id) == keep
    for v, r in enumerate(rows):
        lo, hi = g.row_ptr[v], g.row_ptr[v + 1]
        assert list(zip(g.col[lo:hi].tolist(), g.w[lo:hi].tolist())) == r
    if directed:
        for v in range(g.n):
            lo, hi = g.rrow_ptr[v], g.rrow_ptr[v + 1]
            want = sorted((u, ww) for u, r in enumerate(rows) for (x, ww) in r if x == v)
            assert list(zip(g.rcol[lo:hi].tolist(), g.rw[lo:hi].tolist())) == want


# ---------------------------------------------------------------- estimators

def test_star_example_of_the_introduction():
    gd = golden.read("star_n10.txt")
    n = int(gd["n"][0][0])
    src = [int(x) for x in gd["sources"][0]]
    g = G(synth.star_edges, n)
    assert list(orc.exact_S(g)) == [int(x) for x in gd["S"][0]]
    r1 = orc.estimate(g, src, eps=(1, 1))
    assert r1["pivot"][0] == int(gd["centre_pivot"][0][0])
    assert r1["delta"][0] == int(gd["centre_delta"][0][0])
    assert r1["pivot"][2] == int(gd["leaf_pivot"][0][0])
    assert r1["delta"][2] == int(gd["leaf_delta"][0][0])
    assert list(r1["s_hat"][:3, 0]) == [float(x) for x in gd["centre_s_hat"][0]]
    nd = [int(x) for x in gd["centre_closeness_num_den"][0]]
    for e in range(3):
        assert r1["closeness"][e, 0] == nd[2 * e] / nd[2 * e + 1]
    assert r1["s_hat"][3, 0] == float(gd["centre_hybrid_eps_1_1"][0][0])
    assert list(r1["hyb"][0]) == [int(x) for x in gd["centre_hyb_int_eps_1_1"][0]]
    assert list(r1["s_hat"][:, 2]) == [float(x) for x in gd["leaf_s_hat"][0]]
    r10 = orc.estimate(g, src, eps=(1, 10))
    assert r10["s_hat"][3, 0] == float(gd["centre_hybrid_eps_1_10"][0][0])
    # "almost 100%" error of pivoting and "about three times" of the bound
    big = G(synth.star_edges, 2001)
    rb = orc.estimate(big, [5, 9, 1], eps=(1, 1))
    assert abs(rb["s_hat"][1, 0] / 2000 - 2) < 1e-3
    assert abs(rb["s_hat"][2, 0] / 2000 - 3) < 1e-3


def test_path_hand_evaluation_of_eq4():
    gd = golden.read("path7_eps_half.txt")
    n = int(gd["n"][0][0])
    src = [int(x) for x in gd["sources"][0]]
    eps = tuple(int(x) for x in gd["eps"][0])
    g = G(synth.path_edges, n)
    r = orc.estimate(g, src, eps=eps)
    ints = lambda key: [int(x) for x in gd[key][0]]
    assert list(orc.exact_S(g)) == ints("S")
    assert list(r["pivot"]) == ints("pivot")
    assert list(r["delta"]) == ints("delta")
    assert list(r["sum"]) == ints("sum")
    assert list(r["delta_cc"].ravel()) == ints("delta_cc")
    for e, name in enumerate(orc.EST_NAMES):
        assert list(r["s_hat"][e]) == [float(x) for x in gd["s_hat_" + name][0]]
        assert np.allclose(r["closeness"][e], (n - 1) / r["s_hat"][e], rtol=0)
    for row in gd["hyb"]:
        v = int(row[0])
        assert list(r["hyb"][v]) == [int(x) for x in row[1:]]


def mixed_graphs():
    yield G(synth.grid_edges, 6, 5)
    yield G(synth.rmat_edges, 7, 6, 0.57, 0.19, 0.19, 3)
    n, s, d = synth.watts_strogatz_edges(60, 4, 0.2, seed=4)
    yield orc.csr_from_edges(n, s, d, w=synth.random_weights(s.size, 1, 20, 5))


def test_full_sample_is_exact():
    """C = V: every node is sampled, so every estimator is exact (section 2,
    "for points j in C we can compute the exact value")."""
    for g in mixed_graphs():
        S = orc.exact_S(g)
        r = orc.estimate(g, orc.choose_sample(g.n, g.n, 11), eps=(1, 3))
        for e in range(4):
            assert (r["s_hat"][e] == S.astype(np.float64)).all()
        assert (r["closeness"][3] == orc.exact_closeness(S)).all()


def test_sampled_nodes_exact_and_sample_all_but_one():
    for g in mixed_graphs():
        S = orc.exact_S(g)
        C = orc.choose_sample(g.n, max(2, g.n // 5), 3)
        r = orc.estimate(g, C, eps=(1, 4))
        assert (r["S_samp"] == S[C]).all()
        for e in range(4):
            assert (r["s_hat"][e][C] == S[C]).all()
        # k = n-1 with j unsampled: the sampling estimate is exact
        j = g.n // 2
        C2 = np.array([v for v in range(g.n) if v != j], dtype=np.int32)
        r2 = orc.estimate(g, C2, eps=(1, 4))
        assert r2["s_hat"][0][j] == S[j]


def test_sampling_estimator_is_unbiased_over_all_subsets():
    """E[(n-1)/k * sum_{i in C} d_ij] = S(j) over uniform C of V minus {j}
    (eq. (3)); checked exactly over every k-subset of a small graph."""
    g = G(synth.rmat_edges, 4, 3, 0.57, 0.19, 0.19, 2)
    n = g.n
    S = orc.exact_S(g)
    k, j = 3, 1
    others = [v for v in range(n) if v != j]
    tot, est_tot, cnt = 0, Fraction(0), 0
    for C in itertools.combinations(others, k):
        r = orc.estimate(g, list(C), eps=(1, 2))
        tot += int(r["sum"][j])
        est_tot += Fraction(r["s_hat"][0][j])
        cnt += 1
    assert tot * (n - 1) == k * int(S[j]) * cnt
    assert abs(float(est_tot / cnt) - S[j]) < 1e-9 * S[j]


def test_tiny_eps_reduces_hybrid_to_sampling():
    """eps -> 0 puts every node in L(j) (threshold beyond every distance), so
    eq. (4) becomes the sampling estimate."""
    for g in mixed_graphs():
        C = orc.choose_sample(g.n, 7, 5)
        maxd = int(orc.dist_table(g, C).max())
        r = orc.estimate(g, C, eps=(1, g.n * maxd + 1))
        assert (r["s_hat"][3] == r["s_hat"][0]).all()
        notC = np.setdiff1d(np.arange(g.n), C)
        assert (r["hyb"][notC, 4] == 7).all()  # LCnum = k
        assert (r["hyb"][notC, 1] == 0).all()  # Hnum = 0


def multi_source_first_arrival(g, C):
    """Independent pivot computation: one multi-source search from all of C
    (section 3: "a single run of Dijkstra having all sampled nodes as
    sources"), keyed by (distance, sample index)."""
    INF = (1 << 62)
    best = [(INF, INF)] * g.n
    pq = []
    for i, c in enumerate(C):
        best[c] = (0, i)
        heapq.heappush(pq, (0, i, c))
    done = [False] * g.n
    while pq:
        d, i, u = heapq.heappop(pq)
        if done[u] or (d, i) != best[u]:
            continue
        done[u] = True
        for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
            v = int(g.col[e])
            nd = d + (1 if g.w is None else int(g.w[e]))
            if (nd, i) < best[v]:
                best[v] = (nd, i)
                heapq.heappush(pq, (nd, i, v))
    return [b[1] for b in best], [b[0] for b in best]


def test_pivots_match_multi_source_search():
    for g in mixed_graphs():
        for k in (1, 4, 13):
            C = orc.choose_sample(g.n, k, 9)
            r = orc.estimate(g, C)
            piv, dl = multi_source_first_arrival(g, C)
            assert list(r["pivot"]) == piv and list(r["delta"]) == dl
            s = orc.streaming_pass(g, C)
            assert (s["pivot"] == r["pivot"]).all() and (s["delta"] == r["delta"]).all()
            assert (s["sum"] == r["sum"]).all() and (s["S_samp"] == r["S_samp"]).all()


def test_hybrid_invariants():
    for g in mixed_graphs():
        S = orc.exact_S(g).astype(np.int64)
        k = 9
        C = orc.choose_sample(g.n, k, 21)
        for eps in [(1, 1), (1, 2), (1, 3), (2, 7)]:
            r = orc.estimate(g, C, eps=eps)
            notC = np.setdiff1d(np.arange(g.n), C)
            h = r["hyb"][notC].astype(np.int64)
            Hnum, LCnum = h[:, 1], h[:, 4]
            HCnum = k - LCnum
            assert (LCnum >= 1).all()                      # c(j) in L(j) cap C
            assert ((g.n - 1) - Hnum - HCnum >= LCnum).all()  # |L| >= |L cap C|
            assert (h[:, 2] + h[:, 3] == r["sum"][notC].astype(np.int64)).all()
            # pivot triangle bound: |S(v) - S(c(v))| <= n * Delta(v)
            Sp = S[C[r["pivot"]]]
            assert (np.abs(S - Sp) <= g.n * r["delta"].astype(np.int64)).all()
            # H-part error bound from the proof of Theorem 2.1:
            # each i in H(j) has |d(c(j),i) - d(j,i)| <= Delta(j) and
            # d(j,i) >= Delta(j)(1/eps - 1)
            a, b = eps
            tab = orc.dist_table(g, C)
            for j in notC[:20]:
                p, D = r["pivot"][j], int(r["delta"][j])
                dj = orc.sssp(g, int(j)).astype(np.int64)
                Hset = [w for w in notC if tab[p, w] * a > D * b]
                assert len(Hset) == r["hyb"][j, 1]
                assert sum(int(tab[p, w]) for w in Hset) == r["hyb"][j, 0]
                for w in Hset:
                    assert abs(int(tab[p, w]) - dj[w]) <= D
                    assert dj[w] * a >= D * (b - a)
        if g.w is None:
            assert (r["delta_cc"] == r["delta_cc"].T).all()


def test_roundtrip_estimates_on_directed_cycle_are_exact():
    n = 11
    s = np.arange(n, dtype=np.uint32)
    g = orc.csr_from_edges(n, s, (s + 1) % n, directed=True)
    C = [3, 8, 0]
    r = orc.estimate(g, C, eps=(1, 2), roundtrip=True)
    for e in (0, 1, 3):
        assert (r["s_hat"][e] == n * (n - 1)).all()
    # pivoting upper bound adds (n-1) * Delta = (n-1) * n off the sample
    up = np.where(np.isin(np.arange(n), C), n * (n - 1), 2 * n * (n - 1))
    assert (r["s_hat"][2] == up).all()


def test_exhaustive_tiny_hybrid_against_definition_sets():
    """Every 2-subset of a 7-node graph and several eps: the oracle's integer
    statistics against a literal set evaluation of eq. (4) on Floyd-Warshall
    distances."""
    n, s, d = synth.watts_strogatz_edges(7, 4, 0.3, seed=2)
    g = orc.csr_from_edges(n, s, d)
    D = floyd_warshall(g.n, g.row_ptr, g.col, None)
    for C in itertools.combinations(range(g.n), 2):
        for a, b in [(1, 1), (1, 2), (2, 3)]:
            r = orc.estimate(g, list(C), eps=(a, b))
            for j in range(g.n):
                if j in C:
                    assert r["s_hat"][3][j] == D[j].sum()
                    continue
                dists = [D[c, j] for c in C]
                p = min(range(len(C)), key=lambda i: (dists[i], i))
                Dl = dists[p]
                far = lambda x: x * a > Dl * b
                H = [w for w in range(g.n) if w not in C and far(D[C[p], w])]
                HC = [i for i in range(len(C)) if far(D[C[p], C[i]])]
                LC = [i for i in range(len(C)) if i not in HC]
                L = (g.n - 1) - len(H) - len(HC)
                want = (Fraction(sum(D[C[p], w] for w in H))
                        + sum(D[j, C[i]] for i in HC)
                        + Fraction(L, len(LC)) * sum(D[j, C[i]] for i in LC))
                assert abs(r["s_hat"][3][j] - float(want)) <= 1e-12 * float(want)


@pytest.mark.parametrize("gen,w,k,eps", [
    (lambda: synth.rmat_edges(9, 8, seed=3), None, 40, (1, 6)),
    (lambda: synth.grid_edges(20, 15), None, 12, (1, 2)),
    (lambda: synth.rmat_edges(8, 8, seed=5), "w", 20, (1, 4)),
])
def test_single_node_estimate_equals_table(gen, w, k, eps):
    """The one-node oracle (two searches per node, for graphs too large for
    a k x n table) gives the table oracle's pivot, Delta, sum and all four
    estimates for every node."""
    n, s, d = gen()
    wt = synth.random_weights(s.size, 1, 9, seed=2) if w else None
    g = orc.csr_from_edges(n, s, d, w=wt)
    C = orc.choose_sample(g.n, k, 7)
    ref = orc.estimate_from_table(orc.dist_table(g, C), C, eps)
    for v in range(g.n):
        r = orc.estimate_node(g, C, v, eps)
        assert r["pivot"] == ref["pivot"][v] and r["delta"] == ref["delta"][v]
        assert r["sum"] == int(ref["sum"][v])
        assert r["hyb"] == [int(x) for x in ref["hyb"][v]], v
        for e in range(4):
            assert r["s_hat"][e] == ref["s_hat"][e][v], (v, e)
    p1 = orc.pass1_from_table(orc.dist_table(g, C), C)
    for key in ("pivot", "delta", "sum", "S_samp", "delta_cc"):
        assert (p1[key] == ref[key]).all(), key


@pytest.mark.parametrize("w", [None, "w"])
def test_single_node_round_trip_equals_table(w):
    """Round trips (section 6.1): the one-node oracle's forward and reversed
    searches give the round-trip table oracle's statistics and estimates."""
    n, s, d = synth.rmat_edges(9, 6, seed=13)
    wt = synth.random_weights(s.size, 1, 7, seed=4) if w else None
    g = orc.csr_from_edges(n, s, d, w=wt, directed=True)
    C = orc.choose_sample(g.n, 24, 3)
    ref = orc.estimate_from_table(orc.dist_table(g, C, roundtrip=True), C, (1, 3))
    for v in range(g.n):
        r = orc.estimate_node(g, C, v, (1, 3), roundtrip=True)
        assert r["pivot"] == ref["pivot"][v] and r["delta"] == ref["delta"][v]
        assert r["sum"] == int(ref["sum"][v])
        assert r["hyb"] == [int(x) for x in ref["hyb"][v]], v
        for e in range(4):
            assert r["s_hat"][e] == ref["s_hat"][e][v], (v, e)
