"""GPU parity of the outbound / inbound estimates of general directed graphs
(section 6.2, Algorithm 4) against the oracle: per node the sample count,
the sum of the sample's distances and the rank position T bit-exact, the
average distance and the size estimate within 1e-12 relative.  Covers graphs
with many small and a few large reachability sets (directed R-MAT without
taking a component), a DAG, a cycle, k below, at and above the 64 W-source
group, an undirected graph, several groups per run, and arc lengths
(label-correcting rounds against the oracle's Dijkstra)."""
import numpy as np
import pytest

import synth
from oracle import oracle as orc

pytestmark = pytest.mark.gpu
RTOL = 1e-12


@pytest.fixture(scope="module")
def cc():
    from paper_1409_0035_gb300 import build
    build.build()
    import paper_1409_0035_gb300 as m
    return m


def close(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b) <= RTOL * np.abs(b)


def dag_edges(n, seed):
    # random DAG: arcs from lower to higher id (reach sets of every size)
    rng = np.random.default_rng(seed)
    s = rng.integers(0, n - 1, 4 * n)
    d = s + 1 + rng.integers(0, 40, s.size)
    keep = d < n
    return n, s[keep].astype(np.uint32), d[keep].astype(np.uint32)


GRAPHS = {
    "rmat10-directed": lambda: synth.rmat_edges(10, 6, seed=3),
    "rmat11-directed": lambda: synth.rmat_edges(11, 4, seed=5),
    "dag1500": lambda: dag_edges(1500, 2),
    "cycle300": lambda: (300, np.arange(300, dtype=np.uint32),
                         ((np.arange(300) + 1) % 300).astype(np.uint32)),
}


def check(cc, n, s, d, k, seed, inbound, directed=True, w=None):
    g, _ = cc.cc_graph_from_edges(n, s, d, w, directed=directed, keep_component=False)
    og = orc.csr_from_edges(n, s, d, w=w, directed=directed, keep_component=False)
    try:
        assert cc.cc_graph_info(g)[0] == og.n
        r = cc.cc_reach_estimate(g, k, seed, inbound)
    finally:
        cc.cc_graph_free(g)
    ref = orc.reach_from_table(orc.all_pairs(og), orc.sample_order(og.n, seed), k,
                               inbound=inbound)
    assert np.array_equal(r["count"], ref["count"])
    assert np.array_equal(r["distsum"], ref["distsum"])
    assert np.array_equal(r["T"], ref["T"])
    assert close(r["avg"], ref["avg"]).all()
    assert close(r["R_hat"], ref["R_hat"]).all()
    return r


CASES = [
    ("rmat10-directed", 16, False), ("rmat10-directed", 16, True),
    ("rmat10-directed", 64, False), ("rmat11-directed", 300, True),
    ("rmat11-directed", 2, False), ("dag1500", 8, False), ("dag1500", 8, True),
    ("dag1500", 1, False), ("cycle300", 299, False), ("cycle300", 40, True),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-k{c[1]}-{'in' if c[2] else 'out'}"
                                             for c in CASES])
def test_reach_matches_oracle(cc, case):
    name, k, inbound = case
    n, s, d = GRAPHS[name]()
    r = check(cc, n, s, d, k, seed=7, inbound=inbound)
    assert (r["count"] > 0).any()


def test_undirected_in_and_out_agree(cc):
    n, s, d = synth.watts_strogatz_edges(700, 6, 0.1, seed=4)
    a = check(cc, n, s, d, 12, seed=3, inbound=False, directed=False)
    b = check(cc, n, s, d, 12, seed=3, inbound=True, directed=False)
    assert np.array_equal(a["distsum"], b["distsum"])


WCASES = [
    # graph, k, inbound, arc-length range
    ("rmat10-directed", 16, False, (1, 9)), ("rmat10-directed", 16, True, (1, 9)),
    ("rmat11-directed", 300, False, (1, 1000)), ("dag1500", 8, True, (1, 50)),
    ("cycle300", 299, False, (1, 5)),
]


@pytest.mark.parametrize("case", WCASES, ids=[f"{c[0]}-k{c[1]}-{'in' if c[2] else 'out'}-w"
                                              for c in WCASES])
def test_reach_arc_lengths_match_oracle(cc, case):
    # Section 6.2 runs Dijkstra: with arc lengths the device's
    # label-correcting rounds must give the same samples (reachability does
    # not depend on lengths) and the shortest-path distance sums.
    name, k, inbound, (lo, hi) = case
    n, s, d = GRAPHS[name]()
    w = synth.random_weights(s.size, lo, hi, seed=k)
    r = check(cc, n, s, d, k, seed=5, inbound=inbound, w=w)
    assert (r["count"] > 0).any()


@pytest.mark.parametrize("inbound", [False, True])
def test_reach_group_width_does_not_change_samples(cc, inbound):
    """Groups of 1 to 16 words (64 to 1,024 sources searched together)
    prune at different points but take the same bottom-k samples."""
    n, s, d = synth.rmat_edges(12, 8, seed=31)
    g, _ = cc.cc_graph_from_edges(n, s, d, directed=True, keep_component=False)
    try:
        ref = None
        for words in (1, 2, 4, 8, 16):
            cc.cc_set_param(g, cc.CC_PARAM_REACH_WORDS, words)
            r = cc.cc_reach_estimate(g, 40, 5, inbound)
            if ref is None:
                ref = r
                continue
            for key in ("count", "distsum", "T", "avg", "R_hat"):
                assert (r[key] == ref[key]).all(), (words, key)
    finally:
        cc.cc_graph_free(g)
