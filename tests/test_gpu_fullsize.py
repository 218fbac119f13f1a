"""Full-size parity: every configured workload at the size the benchmark
runs it, through the same C-ABI calls, against the oracle.

Where a k x n distance table fits in host memory (the headline, the road
graphs, the round trips) the oracle's first-pass statistics -- pivot, Delta,
the sum of distances to the sample, exact S of the sampled nodes and the
distances between them -- are compared for every node, bit for bit.  The
estimates, the hybrid's integers and the section 5 / section 6.2 outputs
are compared on picked nodes, each from the oracle's searches out of that
node (and out of its pivot): the highest degrees (hubs), random nodes of
every degree class the traversal treats apart, and sampled nodes.
Integers bit-exact; FP64 within 1e-12 relative."""
import numpy as np
import pytest

import synth
from oracle import oracle as orc
from tests import fullsize as fs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    from paper_1409_0035_gb300 import build
    build.build()
    import paper_1409_0035_gb300 as m
    return m


@pytest.fixture(scope="module")
def rmat20():
    """R-MAT scale 20, edge factor 16, seed 1: the headline graph's edges."""
    return synth.rmat_edges(20, 16, seed=1)


def _check_pass1(r, og, C, roundtrip=False):
    p1 = orc.pass1_from_table(fs.dist_table(og, C, roundtrip), C)
    for key in ("pivot", "delta", "sum", "S_samp", "delta_cc"):
        bad = np.flatnonzero((np.asarray(r[key]) != p1[key]).ravel())
        assert bad.size == 0, f"{key}: {bad.size} entries differ, first at {bad[:5]}"


def _check_nodes(r, og, C, eps, nodes, roundtrip=False):
    refs = fs.pmap(lambda v: orc.estimate_node(og, C, v, eps, roundtrip=roundtrip), nodes)
    for v, ref in zip(nodes, refs):
        assert r["pivot"][v] == ref["pivot"] and r["delta"][v] == ref["delta"], v
        assert int(r["sum"][v]) == ref["sum"], v
        assert [int(x) for x in r["hyb"][v]] == ref["hyb"], v
        for e in range(4):
            got, want = r["s_hat"][e][v], ref["s_hat"][e]
            assert fs.rel_close(got, want), (v, e, got, want)
            assert fs.rel_close(r["closeness"][e][v], (og.n - 1) / want), (v, e)


def test_headline_all_nodes(cc, rmat20):
    """The benchmark's workload and call: R-MAT 20 (646,379 nodes, 15.7 M
    edges), k = 256 from sample seed 2, eps = 1/16, every estimator.
    First-pass statistics on all nodes; estimates and hybrid integers on
    about 200 nodes from every degree class, the 20 largest hubs included."""
    n, s, d = rmat20
    g, _ = cc.cc_graph_from_edges(n, s, d)
    try:
        og = orc.csr_from_edges(n, s, d)
        assert cc.cc_graph_info(g)[:2] == (og.n, og.arcs)
        C = cc.cc_sample_choose(g, 256, 2)
        assert (C == orc.choose_sample(og.n, 256, 2)).all()
        r = cc.cc_estimate(g, C)
    finally:
        cc.cc_graph_free(g)
    _check_pass1(r, og, C)
    nodes = fs.picks(np.diff(og.row_ptr), C, seed=20)
    assert len(nodes) >= 200
    _check_nodes(r, og, C, orc.default_eps(256), nodes)


@pytest.fixture(scope="module")
def road():
    """The road-like random geometric graph of the arc-length workload
    (4,194,304 points, mean degree 2.6 after thinning)."""
    return synth.road_like_edges(4 << 20, seed=1)


@pytest.mark.parametrize("scale", [1e3, 1e6])
def test_road_all_nodes(cc, road, scale):
    """Arc lengths round(scale * Euclidean length) + 1 on the road-like
    graph (3.9 M nodes), k = 64, eps = 1/8: the chunked shortest-path
    path at full size."""
    n, s, d, length = road
    w = synth.edge_lengths_to_weights(length, scale)
    g, _ = cc.cc_graph_from_edges(n, s, d, w)
    try:
        og = orc.csr_from_edges(n, s, d, w=w)
        assert cc.cc_graph_info(g)[:2] == (og.n, og.arcs)
        C = cc.cc_sample_choose(g, 64, 2)
        assert (C == orc.choose_sample(og.n, 64, 2)).all()
        r = cc.cc_estimate(g, C, cc.cc_opts_default(64))
    finally:
        cc.cc_graph_free(g)
    _check_pass1(r, og, C)
    nodes = fs.picks(np.diff(og.row_ptr), C, seed=int(scale) % 97, hubs=8, per_class=25)
    _check_nodes(r, og, C, orc.default_eps(64), nodes)


def test_roundtrip_rmat22_all_nodes(cc):
    """Round trips (section 6.1) on directed R-MAT 22, edge factor 16, its
    largest strongly connected component (1.62 M nodes, 64 M arcs), k =
    128, eps = 1/11: the graph built on the device, the forward and
    reversed traversals, every node's first-pass statistics."""
    n, s, d = synth.rmat_edges(22, 16, seed=1)
    g, old = cc.cc_graph_from_edges(n, s, d, directed=True)
    try:
        og = orc.csr_from_edges(n, s, d, directed=True)
        assert cc.cc_graph_info(g)[:2] == (og.n, og.arcs)
        assert (old == og.old_id).all()
        C = cc.cc_sample_choose(g, 128, 2)
        assert (C == orc.choose_sample(og.n, 128, 2)).all()
        o = cc.cc_opts_default(128)
        o.roundtrip = 1
        r = cc.cc_estimate(g, C, o)
    finally:
        cc.cc_graph_free(g)
    _check_pass1(r, og, C, roundtrip=True)
    deg = np.diff(og.row_ptr) + np.diff(og.rrow_ptr)
    nodes = fs.picks(deg, C, seed=22, hubs=10, per_class=15)
    _check_nodes(r, og, C, orc.default_eps(128), nodes, roundtrip=True)


def test_node_weighted_sampled_nodes(cc, rmat20):
    """Section 5 on the headline graph with the benchmark's Pareto node
    weights, k = 256, eps = 1/16: the weighted sample and tau exactly, the
    sampling and hybrid estimates of S_beta and the weighted closeness on
    picked nodes (hubs, every degree class, certain and uncertain sampled
    nodes)."""
    n, s, d = rmat20
    g, _ = cc.cc_graph_from_edges(n, s, d)
    try:
        og = orc.csr_from_edges(n, s, d)
        beta = synth.pareto_node_weights(og.n, seed=1)
        cc.cc_graph_set_node_weights(g, beta)
        C, tau = cc.cc_sample_varopt(g, 256, 2)
        Cw, tw = orc.sample_varopt(beta, 256, 2)
        assert (C == Cw).all() and tuple(tau) == tuple(tw)
        r = cc.cc_estimate_node_weighted(g, C, tau)
    finally:
        cc.cc_graph_free(g)
    certain = [int(c) for c in C if orc.is_certain(int(beta[c]), tau)]
    nodes = fs.picks(np.diff(og.row_ptr), C, seed=5, hubs=10, per_class=20,
                     extra=certain[:5] + [int(c) for c in C[1:6]])
    eps = orc.default_eps(256)
    refs = fs.pmap(lambda v: orc.node_weighted_node(og, C, beta, tau, v, eps), nodes)
    idx = {int(c): i for i, c in enumerate(C)}
    for v, ref in zip(nodes, refs):
        for e in range(2):
            assert fs.rel_close(r["s_hat"][e][v], ref["s_hat"][e]), (v, e)
            assert fs.rel_close(r["closeness"][e][v], ref["closeness"][e]), (v, e)
        if v in idx:
            assert int(r["S_sampled"][idx[v]]) * tau[1] == ref["num"][0], v


@pytest.mark.parametrize("inbound", [False, True])
def test_reach_sampled_nodes(cc, rmat20, inbound):
    """Section 6.2 on the directed R-MAT 20 graph kept whole (1,048,576
    nodes, half of them without out-arcs), k = 64, order seed 2: count,
    distance sum and T exactly, the average distance and the size estimate
    within 1e-12, on picked nodes (hubs of both directions, every degree
    class, nodes with no arcs)."""
    n, s, d = rmat20
    g, _ = cc.cc_graph_from_edges(n, s, d, directed=True, keep_component=False)
    try:
        og = orc.csr_from_edges(n, s, d, directed=True, keep_component=False)
        r = cc.cc_reach_estimate(g, 64, 2, inbound)
    finally:
        cc.cc_graph_free(g)
    order = orc.sample_order(og.n, 2)
    outd, ind = np.diff(og.row_ptr), np.diff(og.rrow_ptr)
    nodes = fs.picks(ind if inbound else outd, order[:2], seed=7 + inbound, hubs=10,
                     per_class=25, extra=np.argsort(-(outd + ind))[:5])
    refs = fs.pmap(lambda v: orc.reach_node(og, order, v, 64, inbound=inbound), nodes)
    for v, ref in zip(nodes, refs):
        assert r["count"][v] == ref["count"] and int(r["distsum"][v]) == ref["distsum"], v
        assert int(r["T"][v]) == ref["T"], v
        assert fs.rel_close(r["avg"][v], ref["avg"]) or r["avg"][v] == ref["avg"] == 0.0, v
        assert fs.rel_close(r["R_hat"][v], ref["R_hat"]), v
