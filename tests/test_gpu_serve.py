"""Serving with continuous batching: every request's result in a mixed,
overlapping stream equals the same request run alone (bit for bit: the
arithmetic is exact integers plus one rounding), and the server really ran
requests concurrently."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    from paper_1409_0035_gb300 import build
    build.build()
    import paper_1409_0035_gb300 as m
    return m


def test_results_same_alone_and_in_the_mix(cc):
    gens = [synth.rmat_edges(11, 16, seed=1), synth.grid_edges(60, 40),
            synth.watts_strogatz_edges(3000, 10, 0.05, seed=2), synth.rmat_edges(13, 8, seed=3)]
    handles, ns = [], []
    for n, s, d in gens:
        g, _ = cc.cc_graph_from_edges(n, s, d)
        handles.append(g)
        ns.append(cc.cc_graph_info(g)[0])
    reqs = []
    rng = np.random.default_rng(5)
    for i in range(24):
        gi = int(rng.integers(0, len(handles)))
        est = int(rng.integers(0, 4))
        k = int(rng.choice([16, 64, 128, 300]))
        reqs.append((gi, est, min(k, ns[gi]), 100 + i))
    try:
        srv = cc.cc_server_create(handles, slots=4)
        try:
            ids = [cc.cc_server_submit(srv, gi, est, k, seed) for gi, est, k, seed in reqs]
            got = []
            for rid, (gi, est, k, seed) in zip(ids, reqs):
                assert cc.cc_server_wait(srv, rid, 120000) == cc.CC_OK
                got.append(cc.cc_server_result(srv, rid, ns[gi]))
            st = cc.cc_server_stats(srv)
            assert st["completed"] == len(reqs)
            assert st["peak_running"] >= 2  # requests overlapped
            assert st["p99_ms"] >= st["p50_ms"] > 0
        finally:
            cc.cc_server_free(srv)
        for (gi, est, k, seed), r in zip(reqs, got):
            C = cc.cc_sample_choose(handles[gi], k, seed)
            o = cc.cc_opts_default(k)
            o.want_hybrid = int(est == 3)
            alone = cc.cc_estimate(handles[gi], C, o)
            assert (r["s_hat"] == alone["s_hat"][est]).all()
            assert (r["closeness"] == alone["closeness"][est]).all()
            assert (r["pivot"] == alone["pivot"]).all()
            assert (r["delta"] == alone["delta"]).all()
            assert (r["sum"] == alone["sum"]).all()
    finally:
        for g in handles:
            cc.cc_graph_free(g)


def _alone(cc, g, k, seed, est, eps, roundtrip=False):
    C = cc.cc_sample_choose(g, k, seed)
    o = cc.cc_opts_default(k)
    o.eps_num, o.eps_den = eps
    o.want_hybrid = int(est == 3)
    o.roundtrip = int(roundtrip)
    return cc.cc_estimate(g, C, o)


@pytest.mark.parametrize("budget_mb", [0, 12])
def test_resident_sampled_state_is_reused(cc, budget_mb):
    """Requests repeating a (graph, k, seed) sample with other estimators
    and eps values run from its resident first pass (the hybrid's deferred
    bits when the eps matches, its second pass otherwise) and give the same
    answer as a fresh call; a small budget forces evictions, still exact."""
    gens = [(synth.grid_edges(70, 50), None, False),
            (synth.rmat_edges(12, 8, seed=7), None, False),
            (synth.watts_strogatz_edges(2000, 6, 0.05, seed=3),
             synth.random_weights(6000, 1, 20, seed=4), False),
            (synth.rmat_edges(10, 8, seed=11), None, True)]
    handles, ns, dirs = [], [], []
    for (n, s, d), w, directed in gens:
        g, _ = cc.cc_graph_from_edges(n, s, d, w, directed=directed)
        handles.append(g)
        ns.append(cc.cc_graph_info(g)[0])
        dirs.append(directed)
    plan = []
    for rep in range(3):
        for gi in range(len(handles)):
            for est, eps in ((3, (1, 8)), (0, (1, 8)), (3, (1, 3)), (1, (1, 8)), (3, (1, 8))):
                plan.append((gi, est, min(100, ns[gi]), 9, eps))
    try:
        srv = cc.cc_server_create(handles, slots=3, hbm_budget=budget_mb << 20)
        try:
            got = []
            for gi, est, k, seed, eps in plan:  # one at a time: hits are certain
                rid = cc.cc_server_submit(srv, gi, est, k, seed, eps)
                assert cc.cc_server_wait(srv, rid, 120000) == cc.CC_OK
                got.append(cc.cc_server_result(srv, rid, ns[gi]))
            cs = cc.cc_server_cache_stats(srv)
            assert cs["hits"] + cs["misses"] == len(plan)
            if budget_mb == 0:
                assert cs["misses"] == len(handles) and cs["hits"] == len(plan) - len(handles)
            else:
                assert cs["misses"] > len(handles)  # evictions forced re-runs
        finally:
            cc.cc_server_free(srv)
        for (gi, est, k, seed, eps), r in zip(plan, got):
            alone = _alone(cc, handles[gi], k, seed, est, eps, dirs[gi])
            assert (r["s_hat"] == alone["s_hat"][est]).all(), (gi, est, eps)
            assert (r["pivot"] == alone["pivot"]).all()
            assert (r["sum"] == alone["sum"]).all()
    finally:
        for g in handles:
            cc.cc_graph_free(g)
