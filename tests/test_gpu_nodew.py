"""GPU parity of node-weighted closeness (section 5, "Weighted Centrality")
against the oracle: the weighted sample and its threshold bit-exact, the exact
S_beta of the sampled nodes bit-exact, the sampling and hybrid estimates and
the weighted closeness within 1e-12 relative (each is one integer numerator,
at most two roundings, against the oracle's exact fraction rounded once).
Covers unit and arc lengths, round trips, more than one chunk of sources
with a ragged last slice, zero weights and a sample of every positive
weight."""
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


def weights(n, kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "unit":
        return np.ones(n, np.uint32)
    if kind == "uniform":
        return rng.integers(1, 100, n).astype(np.uint32)
    if kind == "heavy":  # Pareto-like: a few nodes carry much of the weight
        return np.minimum(np.floor(rng.pareto(1.2, n) * 10) + 1, 1e6).astype(np.uint32)
    if kind == "zeros":
        b = rng.integers(1, 20, n).astype(np.uint32)
        b[rng.random(n) < 0.5] = 0
        return b
    raise ValueError(kind)


def close(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b) <= RTOL * np.abs(b)


def build_pair(cc, gen, wlen, directed):
    n, s, d = gen()
    w = synth.random_weights(s.size, 1, 9, seed=8) if wlen else None
    g, _ = cc.cc_graph_from_edges(n, s, d, w, directed=directed, keep_component=True)
    og = orc.csr_from_edges(n, s, d, w=w, directed=directed, keep_component=True)
    assert cc.cc_graph_info(g)[0] == og.n
    return g, og


GRAPHS = {
    "rmat10": (lambda: synth.rmat_edges(10, 8, seed=3), False, False),
    "grid40x30": (lambda: synth.grid_edges(40, 30), False, False),
    "ws900": (lambda: synth.watts_strogatz_edges(900, 10, 0.05, seed=6), False, False),
    "rmat10-lengths": (lambda: synth.rmat_edges(10, 8, seed=7), True, False),
    "rmat9-roundtrip": (lambda: synth.rmat_edges(9, 8, seed=9), False, True),
    "rmat9-roundtrip-lengths": (lambda: synth.rmat_edges(9, 8, seed=9), True, True),
}


@pytest.mark.parametrize("kind,k,seed", [("unit", 64, 1), ("uniform", 7, 2), ("heavy", 200, 3),
                                         ("zeros", 33, 4), ("heavy", 1, 5)])
def test_sample_matches_oracle(cc, kind, k, seed):
    g, og = build_pair(cc, *GRAPHS["rmat10"])
    try:
        beta = weights(og.n, kind, seed)
        cc.cc_graph_set_node_weights(g, beta)
        C, tau = cc.cc_sample_varopt(g, k, seed)
    finally:
        cc.cc_graph_free(g)
    C0, tau0 = orc.sample_varopt(beta, k, seed)
    assert tau == tau0
    assert np.array_equal(C, C0)


def test_sample_of_every_positive_weight(cc):
    g, og = build_pair(cc, *GRAPHS["grid40x30"])
    try:
        beta = np.zeros(og.n, np.uint32)
        pos = np.random.default_rng(3).choice(og.n, 25, replace=False)
        beta[pos] = np.arange(1, 26)
        cc.cc_graph_set_node_weights(g, beta)
        C, tau = cc.cc_sample_varopt(g, 25, 9)
        assert sorted(C.tolist()) == sorted(pos.tolist())
        assert tau == orc.sample_varopt(beta, 25, 9)[1]
        r = cc.cc_estimate_node_weighted(g, C, tau)
    finally:
        cc.cc_graph_free(g)
    ref = orc.node_weighted_from_table(orc.dist_table(og, C), C, beta, tau,
                                       orc.default_eps(25))
    # every estimate is exact here
    for e in (0, 1):
        assert close(r["s_hat"][e], ref["s_hat"][e]).all()


CASES = [
    # graph, weight kind, k, eps
    ("rmat10", "heavy", 64, (1, 8)),
    ("rmat10", "unit", 100, (1, 10)),
    ("grid40x30", "uniform", 48, (1, 2)),
    ("ws900", "zeros", 130, (1, 4)),     # two chunks, ragged last slice
    ("rmat10-lengths", "heavy", 70, (1, 3)),
    ("rmat9-roundtrip", "uniform", 40, (1, 2)),
    ("rmat9-roundtrip-lengths", "heavy", 33, (1, 5)),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-{c[1]}-k{c[2]}" for c in CASES])
def test_estimates_match_oracle(cc, case):
    name, kind, k, eps = case
    gen, wlen, directed = GRAPHS[name]
    g, og = build_pair(cc, gen, wlen, directed)
    try:
        beta = weights(og.n, kind, k)
        cc.cc_graph_set_node_weights(g, beta)
        C, tau = cc.cc_sample_varopt(g, k, 17)
        o = cc.cc_opts_default(k)
        o.eps_num, o.eps_den, o.roundtrip = eps[0], eps[1], int(directed)
        r = cc.cc_estimate_node_weighted(g, C, tau, o)
    finally:
        cc.cc_graph_free(g)
    T = orc.dist_table(og, C, roundtrip=directed)
    ref = orc.node_weighted_from_table(T, C, beta, tau, eps)
    assert [int(x) for x in r["S_sampled"]] == ref["S_samp"]
    for e in (0, 1):
        bad = ~close(r["s_hat"][e], ref["s_hat"][e])
        assert not bad.any(), (e, np.flatnonzero(bad)[:5], r["s_hat"][e][bad][:5],
                               ref["s_hat"][e][bad][:5])
        assert close(r["closeness"][e], ref["closeness"][e]).all()


def test_sampling_only_and_device_outputs(cc):
    torch = pytest.importorskip("torch")
    g, og = build_pair(cc, *GRAPHS["rmat10"])
    try:
        beta = weights(og.n, "uniform", 5)
        cc.cc_graph_set_node_weights(g, beta)
        C, tau = cc.cc_sample_varopt(g, 90, 6)
        o = cc.cc_opts_default(90)
        host = cc.cc_estimate_node_weighted(g, C, tau, o)
        o.want_hybrid = 0
        only = cc.cc_estimate_node_weighted(g, C, tau, o)
        o.want_hybrid, o.device_outputs = 1, 1
        dev = [torch.zeros(og.n, dtype=torch.float64, device="cuda") for _ in range(4)]
        Sd = torch.zeros(90, dtype=torch.int64, device="cuda")
        w = cc.cc_wout()
        for e in range(2):
            w.s_hat[e] = dev[2 * e].data_ptr()
            w.closeness[e] = dev[2 * e + 1].data_ptr()
        w.S_sampled = Sd.data_ptr()
        cc.cc_estimate_node_weighted(g, C, tau, o, out=w)
        torch.cuda.synchronize()
    finally:
        cc.cc_graph_free(g)
    assert np.array_equal(only["s_hat"][0], host["s_hat"][0])
    assert not only["s_hat"][1].any()
    for e in range(2):
        assert np.array_equal(dev[2 * e].cpu().numpy(), host["s_hat"][e])
        assert np.array_equal(dev[2 * e + 1].cpu().numpy(), host["closeness"][e])
    assert np.array_equal(Sd.cpu().numpy().astype(np.uint64), host["S_sampled"])


def test_argument_errors(cc):
    g, og = build_pair(cc, *GRAPHS["grid40x30"])
    try:
        with pytest.raises(cc.CCError):  # no weights attached
            cc.cc_sample_varopt(g, 4, 1)
        beta = np.zeros(og.n, np.uint32)
        beta[:3] = 5
        cc.cc_graph_set_node_weights(g, beta)
        with pytest.raises(cc.CCError):  # fewer positive weights than k
            cc.cc_sample_varopt(g, 4, 1)
        with pytest.raises(cc.CCError):  # a sampled node of weight 0
            cc.cc_estimate_node_weighted(g, np.array([0, 1, 2, 3], np.int32), (15, 4))
        with pytest.raises(cc.CCError):  # tau = 0
            cc.cc_estimate_node_weighted(g, np.array([0, 1, 2], np.int32), (0, 1))
        cc.cc_graph_set_node_weights(g, None)
        with pytest.raises(cc.CCError):  # detached
            cc.cc_estimate_node_weighted(g, np.array([0, 1, 2], np.int32), (5, 1))
    finally:
        cc.cc_graph_free(g)
