"""Pins of the oracle's node-weighted closeness (section 5, "Weighted
Centrality"): the threshold tau, the exact-size weighted sample and the
sampling and hybrid estimates of S_beta.

Each pin checks a property the section fixes rather than re-evaluating the
oracle's own formulas: tau solves sum min(1, beta/tau) = k; over every
offset of the systematic draw each node is picked with probability
min(1, beta/tau) and the inverse-probability estimate averages to the exact
S_beta (scipy's all-pairs shortest paths, a library routine, gives S_beta);
unit weights reduce to the unweighted oracle; a sample holding every
positive weight is exact; and a small path is worked by hand.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

import synth
from oracle import oracle as O


def _apsp(g):
    """n x n distances by scipy (unit lengths when the graph has none)."""
    w = np.ones(g.arcs) if g.w is None else g.w.astype(np.float64)
    A = sp.csr_matrix((w, g.col, g.row_ptr), shape=(g.n, g.n))
    D = shortest_path(A, directed=True, unweighted=g.w is None)
    assert np.isfinite(D).all()
    return D.astype(np.int64)


def _weights(n, kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        return rng.integers(1, 10, n)
    if kind == "heavy":  # a few very heavy nodes among light ones
        b = rng.integers(1, 4, n)
        b[rng.choice(n, max(1, n // 8), replace=False)] = rng.integers(50, 400, max(1, n // 8))
        return b
    if kind == "zeros":
        b = rng.integers(0, 6, n)
        b[rng.random(n) < 0.4] = 0
        return b
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["uniform", "heavy", "zeros"])
@pytest.mark.parametrize("k", [1, 3, 7, 20])
def test_threshold_solves_its_equation(kind, k):
    beta = _weights(40, kind, seed=k)
    if (beta > 0).sum() < k:
        pytest.skip("fewer positive weights than k")
    tn, td = O.varopt_threshold(beta, k)
    tau = Fraction(tn, td)
    total = sum(min(Fraction(1), Fraction(int(b)) / tau) for b in beta if b > 0)
    if (beta > 0).sum() == k:
        assert all(b >= tau for b in beta if b > 0)  # every positive weight certain
    else:
        assert total == k
    for b in beta:
        assert O.is_certain(int(b), (tn, td)) == (b > 0 and b >= tau) or b == 0


def test_threshold_closed_forms():
    # unit weights: tau = n / k; 0/1 weights: tau = (number of ones) / k
    assert Fraction(*O.varopt_threshold([1] * 30, 4)) == Fraction(30, 4)
    b = [1, 0, 1, 1, 0, 1, 1, 0, 0, 1]
    assert Fraction(*O.varopt_threshold(b, 2)) == Fraction(6, 2)
    # one dominant weight: certain, the rest share k - 1 draws
    assert O.varopt_threshold([100, 1, 1, 1, 1], 2) == (4, 1)


@pytest.mark.parametrize("kind", ["uniform", "heavy", "zeros"])
def test_systematic_draw_has_exact_marginals(kind):
    # Every offset u in [0, tn) of one random order: node v is picked for
    # beta(v) * td offsets (probability beta/tau), certain nodes for all,
    # zero weights for none, and every draw has exactly k nodes.
    n, k = 14, 5
    beta = _weights(n, kind, seed=3)
    tn, td = O.varopt_threshold(beta, k)
    order = O.sample_order(n, 11)
    hits = np.zeros(n, dtype=np.int64)
    for u in range(tn):
        C = O.systematic_pick(order, beta, (tn, td), u)
        assert len(C) == k and len(set(C)) == k
        hits[C] += 1
    for v in range(n):
        b = int(beta[v])
        if b == 0:
            assert hits[v] == 0
        elif O.is_certain(b, (tn, td)):
            assert hits[v] == tn
        else:
            assert hits[v] == b * td


@pytest.mark.parametrize("graph", ["path", "weighted"])
def test_inverse_probability_estimate_is_unbiased(graph):
    # Averaged over every offset u, sum over c in C of max(tau, beta(c))
    # d(c, v) equals S_beta(v) exactly, for every node v; the oracle's
    # sampling estimate of a non-sampled node is that sum.
    if graph == "path":
        g = O.csr_from_edges(*synth.path_edges(9))
    else:
        n, s, d = synth.watts_strogatz_edges(12, 4, 0.3, seed=5)
        g = O.csr_from_edges(n, s, d, w=synth.random_weights(s.size, 1, 6, seed=6))
    n, k = g.n, 3
    beta = _weights(n, "heavy", seed=4)
    beta[0] = 0
    D = _apsp(g)
    S = (D * beta[None, :]).sum(axis=1)
    tn, td = O.varopt_threshold(beta, k)
    tau = Fraction(tn, td)
    order = O.sample_order(n, 2)
    acc = [Fraction(0)] * n
    for u in range(tn):
        C = O.systematic_pick(order, beta, (tn, td), u)
        T = D[C, :]
        r = O.node_weighted_from_table(T, C, beta, (tn, td), (1, 2))
        for v in range(n):
            ht = sum(max(tau, Fraction(int(beta[c]))) * int(D[c, v]) for c in C)
            acc[v] += ht
            if v not in C:
                assert Fraction(r["num"][0][v], td) == ht
    for v in range(n):
        assert acc[v] / tn == S[v], v


def test_unit_weights_reduce_to_the_unweighted_estimates():
    # beta = 1: tau = n/k, so the sampling estimate is n/(n-1) times eq. (3)'s
    # and the hybrid is Hsum + HCsum + (n/k) LCsum of the unweighted
    # accumulators (eq. (4) with the inverse-probability L part).
    g = O.csr_from_edges(*synth.rmat_edges(8, 8, seed=3))
    n, k = g.n, 17
    C = O.choose_sample(n, k, 5)
    T = O.dist_table(g, C)
    beta = np.ones(n, dtype=np.int64)
    tau = O.varopt_threshold(beta, k)
    assert Fraction(*tau) == Fraction(n, k)
    w = O.node_weighted_from_table(T, C, beta, tau, (1, 4))
    u = O.estimate_from_table(T, C, (1, 4))
    Cs = set(C.tolist())
    for v in range(n):
        if v in Cs:
            assert w["num"][0][v] == int(u["S_samp"][C.tolist().index(v)]) * tau[1]
            continue
        assert w["s_hat"][0][v] == pytest.approx(n / (n - 1) * u["s_hat"][0][v], rel=1e-15)
        Hsum, _, HCsum, LCsum, _, _ = (int(x) for x in u["hyb"][v])
        assert Fraction(w["num"][1][v], tau[1]) == Hsum + HCsum + Fraction(n, k) * LCsum


@pytest.mark.parametrize("graph", ["grid", "weighted"])
def test_sample_of_every_positive_weight_is_exact(graph):
    if graph == "grid":
        g = O.csr_from_edges(*synth.grid_edges(6, 5))
    else:
        n, s, d = synth.rmat_edges(6, 6, seed=8)
        g = O.csr_from_edges(n, s, d, w=synth.random_weights(s.size, 1, 9, seed=9))
    n = g.n
    beta = np.zeros(n, dtype=np.int64)
    pos = np.random.default_rng(1).choice(n, 7, replace=False)
    beta[pos] = [3, 1, 4, 1, 5, 9, 2]
    C, tau = O.sample_varopt(beta, 7, seed=3)
    assert sorted(C.tolist()) == sorted(pos.tolist())
    D = _apsp(g)
    S = (D * beta[None, :]).sum(axis=1)
    r = O.node_weighted_from_table(D[C, :], C, beta, tau, (1, 3))
    for row in (0, 1):
        assert [Fraction(x, tau[1]) for x in r["num"][row]] == [Fraction(int(s)) for s in S]
    tot = beta.sum()
    assert np.allclose(r["closeness"][1], (tot - beta) / S, rtol=1e-15)


def test_hand_worked_path():
    # Path 0-1-2-3-4-5, beta = (2, 1, 1, 1, 1, 2), k = 2: tau = 8/2 (no
    # weight reaches 4), so both sampled nodes count 4 d.  C = {0, 5},
    # eps = 1/2 (x beyond when x > 2 Delta).
    #  v = 2: pivot 0, Delta 2; no non-sampled node lies beyond 4 from 0;
    #    node 5 (at 5 from 0) is in HC: 2 * d(5, 2) = 6; L: 4 * d(0, 2) = 8;
    #    hybrid 14 (= S_beta(2) = 4+1+1+2+6); sampling 4*2 + 4*3 = 20.
    #  v = 4: pivot 5, Delta 1; beyond 2 from 5: nodes 1 (4), 2 (3) -> H sum
    #    4 + 3 = 7; node 0 (at 5 from 5) in HC: 2 * d(0, 4) = 8; L: 4 * 1;
    #    hybrid 19; sampling 4*4 + 4*1 = 20.
    #  v = 0 (sampled): S_beta(0) = 1 + 2 + 3 + 4 + 2*5 = 20.
    beta = [2, 1, 1, 1, 1, 2]
    tau = O.varopt_threshold(beta, 2)
    assert Fraction(*tau) == 4
    g = O.csr_from_edges(*synth.path_edges(6))
    C = [0, 5]
    r = O.node_weighted_from_table(O.dist_table(g, np.int32(C)), C, beta, tau, (1, 2))
    assert r["s_hat"][1][2] == 14 and r["s_hat"][0][2] == 20
    assert r["s_hat"][1][4] == 19 and r["s_hat"][0][4] == 20
    assert r["s_hat"][0][0] == r["s_hat"][1][0] == 20
    assert r["S_samp"] == [20, 2 * 5 + 1 * 4 + 1 * 3 + 1 * 2 + 1 * 1]
    assert r["closeness"][1][2] == pytest.approx(7 / 14, rel=1e-15)


@pytest.mark.parametrize("seed", range(6))
def test_sample_is_exact_size_and_skips_zero_weights(seed):
    beta = _weights(60, "zeros", seed=seed)
    beta[:3] = 1000  # certain
    C, tau = O.sample_varopt(beta, 9, seed)
    assert len(C) == 9 and len(set(C.tolist())) == 9
    assert all(beta[c] > 0 for c in C)
    assert {0, 1, 2} <= set(C.tolist())
    order = O.sample_order(60, seed).tolist()
    pos = [order.index(c) for c in C]
    assert pos == sorted(pos)  # listed in the order of the draw


@pytest.mark.parametrize("graph", ["rmat", "weighted", "roundtrip"])
def test_single_node_weighted_equals_table(graph):
    # Two searches per node (from it and from its pivot) give the table
    # function's numerators, estimates and closeness for every node.
    if graph == "roundtrip":
        n, s, d = synth.rmat_edges(8, 6, seed=41)
        g = O.csr_from_edges(n, s, d, directed=True)
    else:
        n, s, d = synth.rmat_edges(8, 6, seed=42)
        w = synth.random_weights(s.size, 1, 9, seed=43) if graph == "weighted" else None
        g = O.csr_from_edges(n, s, d, w=w)
    rt = graph == "roundtrip"
    beta = _weights(g.n, "heavy", seed=44)
    C, tau = O.sample_varopt(beta, 15, seed=45)
    ref = O.node_weighted_from_table(O.dist_table(g, C, roundtrip=rt), C, beta, tau, (1, 3))
    for v in range(g.n):
        r = O.node_weighted_node(g, C, beta, tau, v, (1, 3), roundtrip=rt)
        assert r["num"] == [ref["num"][0][v], ref["num"][1][v]]
        assert r["s_hat"] == [ref["s_hat"][0][v], ref["s_hat"][1][v]]
