"""GPU parity of the hybrid's error estimate SqErrEst (Algorithm 1's last
loop; section 4) against the oracle, on the bit-packed BFS path and on the
chunked shortest-path path (weighted graphs, round trips).  The integer
inputs are exact on both sides and each term is one 128-bit numerator, one
conversion and one division, so the tolerance is the FP64 one of every
other estimate: 1e-12 relative."""
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


def run(cc, n, s, d, w, directed, k, eps, seed=2):
    g, _ = cc.cc_graph_from_edges(n, s, d, w, directed=directed, keep_component=True)
    og = orc.csr_from_edges(n, s, d, w=w, directed=directed, keep_component=True)
    try:
        C = orc.choose_sample(og.n, k, seed)
        o = cc.cc_opts_default(k)
        o.eps_num, o.eps_den, o.want_hybrid = eps[0], eps[1], 1
        o.roundtrip = int(directed)
        r = cc.cc_estimate(g, C, o, want_sqerr=True)
        T = orc.dist_table(og, C, roundtrip=directed)
        s_hat, se = orc.sqerr_from_table(T, C, eps)
        return r, s_hat, se
    finally:
        cc.cc_graph_free(g)


def close(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b) <= RTOL * np.abs(b)


CASES = [
    # name, edge generator, weights, directed, k, eps
    ("rmat10 k=64 eps=1/8", lambda: synth.rmat_edges(10, 8, seed=3), None, False, 64, (1, 8)),
    ("rmat10 k=100 eps=99/100", lambda: synth.rmat_edges(10, 8, seed=4), None, False, 100,
     (99, 100)),
    ("rmat11 k=257 eps=1/2", lambda: synth.rmat_edges(11, 8, seed=5), None, False, 257, (1, 2)),
    ("grid 40x30 k=48 eps=1/2", lambda: synth.grid_edges(40, 30), None, False, 48, (1, 2)),
    ("grid 40x30 k=48 eps=1/5", lambda: synth.grid_edges(40, 30), None, False, 48, (1, 5)),
    ("path 400 k=9 eps=1/3", lambda: synth.path_edges(400), None, False, 9, (1, 3)),
    ("ws 900 k=130 eps=1/4", lambda: synth.watts_strogatz_edges(900, 10, 0.05, seed=6), None,
     False, 130, (1, 4)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_sqerr_bfs_matches_oracle(cc, case):
    _, gen, w, directed, k, eps = case
    n, s, d = gen()
    r, s_hat, se = run(cc, n, s, d, w, directed, k, eps)
    assert close(r["s_hat"][3], s_hat).all()
    bad = ~close(r["sq_err"], se)
    assert not bad.any(), (np.flatnonzero(bad)[:5], r["sq_err"][bad][:5], se[bad][:5])
    assert (se > 0).any()


@pytest.mark.parametrize("eps", [(1, 8), (1, 2), (9, 10)])
def test_sqerr_weighted_matches_oracle(cc, eps):
    n, s, d = synth.rmat_edges(10, 8, seed=7)
    w = synth.random_weights(s.size, 1, 9, seed=8)
    r, s_hat, se = run(cc, n, s, d, w, False, 70, eps)
    assert close(r["s_hat"][3], s_hat).all()
    assert close(r["sq_err"], se).all()


@pytest.mark.parametrize("weighted", [False, True])
def test_sqerr_roundtrip_matches_oracle(cc, weighted):
    n, s, d = synth.rmat_edges(10, 8, seed=9)
    w = synth.random_weights(s.size, 1, 5, seed=10) if weighted else None
    r, s_hat, se = run(cc, n, s, d, w, True, 40, (1, 2))
    assert close(r["s_hat"][3], s_hat).all()
    assert close(r["sq_err"], se).all()


def test_sqerr_full_sample_is_zero(cc):
    n, s, d = synth.cycle_edges(64)
    r, _, se = run(cc, n, s, d, None, False, 64, (1, 2))
    assert not r["sq_err"].any() and not se.any()


ADAPTIVE_CASES = [
    ("rmat10 k=64", lambda: synth.rmat_edges(10, 8, seed=3), None, False, 64),
    ("grid 36x28 k=40", lambda: synth.grid_edges(36, 28), None, False, 40),
    ("ws 800 k=100", lambda: synth.watts_strogatz_edges(800, 10, 0.05, seed=6), None, False,
     100),
    ("rmat9 weighted k=50", lambda: synth.rmat_edges(9, 8, seed=7), "w", False, 50),
    ("rmat9 round trips k=30", lambda: synth.rmat_edges(9, 8, seed=9), None, True, 30),
]


@pytest.mark.parametrize("case", ADAPTIVE_CASES, ids=[c[0] for c in ADAPTIVE_CASES])
def test_adaptive_matches_oracle(cc, case):
    """Adaptive hybrid (section 6) over the paper's eps list: the chosen eps
    bit-exact, estimate and error within 1e-12."""
    _, gen, wkind, directed, k = case
    n, s, d = gen()
    w = synth.random_weights(s.size, 1, 9, seed=8) if wkind else None
    g, _ = cc.cc_graph_from_edges(n, s, d, w, directed=directed, keep_component=True)
    og = orc.csr_from_edges(n, s, d, w=w, directed=directed, keep_component=True)
    try:
        C = orc.choose_sample(og.n, k, 2)
        o = cc.cc_opts_default(k)
        o.roundtrip = int(directed)
        r = cc.cc_estimate_adaptive(g, C, o)
    finally:
        cc.cc_graph_free(g)
    T = orc.dist_table(og, C, roundtrip=directed)
    s_hat, se, choice = orc.adaptive_from_table(T, C)
    assert (r["choice"] == choice).all()
    assert close(r["s_hat"], s_hat).all()
    assert close(r["sq_err"], se).all()
    assert close(r["closeness"], (og.n - 1) / s_hat).all()
    assert len(set(choice[choice >= 0].tolist())) >= 2  # more than one eps wins somewhere


def test_adaptive_custom_list_single_eps_is_fixed_hybrid(cc):
    """A one-entry list is the fixed-eps hybrid with its error estimate."""
    n, s, d = synth.rmat_edges(10, 8, seed=11)
    g, _ = cc.cc_graph_from_edges(n, s, d, keep_component=True)
    try:
        C = orc.choose_sample(cc.cc_graph_info(g)[0], 80, 4)
        ad = cc.cc_estimate_adaptive(g, C, eps_list=[(1, 3)])
        o = cc.cc_opts_default(80)
        o.eps_num, o.eps_den = 1, 3
        fx = cc.cc_estimate(g, C, o, want_sqerr=True)
    finally:
        cc.cc_graph_free(g)
    assert np.array_equal(ad["s_hat"], fx["s_hat"][3])
    assert np.array_equal(ad["sq_err"], fx["sq_err"])
