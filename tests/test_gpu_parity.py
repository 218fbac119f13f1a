"""GPU parity: every output of the sm_103a library against the CPU oracle
on the same seeded inputs.  Integers bit-exact; FP64 within 1e-12 relative
(the arithmetic is the same integer numerator, one conversion and one IEEE
division on both sides)."""
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


def both(cc, n, s, d, w=None, directed=False, keep=True):
    g, old = cc.cc_graph_from_edges(n, s, d, w, directed=directed, keep_component=keep)
    og = orc.csr_from_edges(n, s, d, w=w, directed=directed, keep_component=keep)
    return g, old, og


def assert_close(a, b, what):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    rel = np.abs(a - b) / np.maximum(np.abs(b), 1e-300)
    assert rel.max(initial=0.0) <= RTOL, f"{what}: max rel {rel.max()}"


def check_estimate(cc, g, og, C, eps, hybrid=True):
    o = cc.cc_opts_default(len(C))
    o.eps_num, o.eps_den, o.want_hybrid = eps[0], eps[1], int(hybrid)
    r = cc.cc_estimate(g, C, o)
    want = orc.estimate(og, C, eps=eps)
    assert (r["pivot"] == want["pivot"]).all()
    assert (r["delta"] == want["delta"]).all()
    assert (r["sum"] == want["sum"]).all()
    assert (r["S_samp"] == want["S_samp"]).all()
    assert (r["delta_cc"] == want["delta_cc"]).all()
    nest = 4 if hybrid else 3
    for e in range(nest):
        assert_close(r["s_hat"][e], want["s_hat"][e], f"s_hat[{e}]")
        assert_close(r["closeness"][e], want["closeness"][e], f"closeness[{e}]")
    if hybrid:
        assert (r["hyb"] == want["hyb"]).all()
    return r, want


GRAPHS = {
    "rmat9": lambda: synth.rmat_edges(9, 8, seed=3),
    "grid": lambda: synth.grid_edges(23, 17),
    "ws": lambda: synth.watts_strogatz_edges(700, 10, 0.05, seed=4),
    "path": lambda: synth.path_edges(300),
    "star": lambda: synth.star_edges(1500),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_graph_build_matches_oracle(cc, name):
    n, s, d = GRAPHS[name]()
    g, old, og = both(cc, n, s, d)
    try:
        rp, col, _ = cc.cc_graph_copy_csr(g)
        assert (rp == og.row_ptr).all() and (col == og.col).all()
        assert (old == og.old_id).all()
    finally:
        cc.cc_graph_free(g)


@pytest.mark.parametrize("scale,ef,weighted", [(16, 16, False), (17, 8, True), (14, 4, False)])
def test_graph_build_large_matches_oracle(cc, scale, ef, weighted):
    """Device CSR build (radix sort over many tiles, multi-level scans,
    union-find) against the oracle's numpy build."""
    n, s, d = synth.rmat_edges(scale, ef, seed=scale)
    w = synth.random_weights(s.size, 1, 7, seed=3) if weighted else None
    g, old, og = both(cc, n, s, d, w)
    try:
        rp, col, ww = cc.cc_graph_copy_csr(g)
        assert (rp == og.row_ptr).all() and (col == og.col).all()
        assert (old == og.old_id).all()
        if weighted:
            assert (ww == og.w).all()
    finally:
        cc.cc_graph_free(g)
    g, old = cc.cc_graph_from_edges(n, s, d, w, keep_component=False)
    og = orc.csr_from_edges(n, s, d, w=w, keep_component=False)
    try:
        rp, col, ww = cc.cc_graph_copy_csr(g)
        assert (rp == og.row_ptr).all() and (col == og.col).all()
        assert (old == np.arange(n)).all()
    finally:
        cc.cc_graph_free(g)


def test_graph_build_weighted_directed(cc):
    n, s, d = synth.rmat_edges(9, 6, seed=8)
    w = synth.random_weights(s.size, 1, 30, seed=9)
    for directed in (False, True):
        g, old, og = both(cc, n, s, d, w, directed=directed)
        try:
            rp, col, ww = cc.cc_graph_copy_csr(g)
            assert (rp == og.row_ptr).all() and (col == og.col).all()
            assert (ww == og.w).all() and (old == og.old_id).all()
            if directed:
                rp, col, ww = cc.cc_graph_copy_csr(g, reverse=True)
                assert (rp == og.rrow_ptr).all() and (col == og.rcol).all()
                assert (ww == og.rw).all()
        finally:
            cc.cc_graph_free(g)


def _check_directed_build(cc, n, s, d, w=None, keep=True):
    g, old, og = both(cc, n, s, d, w, directed=True, keep=keep)
    try:
        for rev, (orp, ocol, ow) in ((False, (og.row_ptr, og.col, og.w)),
                                     (True, (og.rrow_ptr, og.rcol, og.rw))):
            rp, col, ww = cc.cc_graph_copy_csr(g, reverse=rev)
            assert (rp == orp).all() and (col == ocol).all()
            if w is not None:
                assert (ww == ow).all()
        assert (old == og.old_id).all()
    finally:
        cc.cc_graph_free(g)


@pytest.mark.parametrize("scale,ef,weighted", [(14, 16, False), (15, 8, True)])
def test_directed_build_device_scc(cc, scale, ef, weighted):
    """Directed R-MAT: merged arcs, G and G^T and the largest strongly
    connected component (a majority component: found on the device)."""
    n, s, d = synth.rmat_edges(scale, ef, seed=scale + 3)
    w = synth.random_weights(s.size, 1, 50, seed=4) if weighted else None
    _check_directed_build(cc, n, s, d, w)


def test_directed_build_without_majority_component(cc):
    """Two directed 40-cycles joined by a 30-node path: the largest
    components tie (the one holding node 0 wins) and none holds half the
    nodes."""
    c1 = synth.cycle_edges(40)
    a = np.concatenate([c1[1], c1[1] + 70, np.arange(40, 69, dtype=np.uint32), [39]])
    b = np.concatenate([c1[2], c1[2] + 70, np.arange(41, 70, dtype=np.uint32), [40]])
    a = np.append(a, np.uint32(69))
    b = np.append(b, np.uint32(70))
    _check_directed_build(cc, 110, a.astype(np.uint32), b.astype(np.uint32))


@pytest.mark.parametrize("scale,ef,weighted", [(18, 16, False), (18, 8, True), (12, 4, False)])
def test_directed_build_minority_scc(cc, scale, ef, weighted):
    """Directed R-MAT with many isolated and one-way nodes: the largest
    strongly connected component holds well under half of the ids (37-47 %),
    so the decomposition has to settle every other part first."""
    n, s, d = synth.rmat_edges(scale, ef, seed=scale + 5)
    w = synth.random_weights(s.size, 1, 50, seed=6) if weighted else None
    _check_directed_build(cc, n, s, d, w)


def _cat(*pairs):
    a = np.concatenate([np.asarray(p[0], np.int64) for p in pairs])
    b = np.concatenate([np.asarray(p[1], np.int64) for p in pairs])
    return a.astype(np.uint32), b.astype(np.uint32)


def _cycle(ids):
    ids = np.asarray(ids, np.int64)
    return ids, np.roll(ids, -1)


def test_directed_build_pivot_in_small_component(cc):
    """The node of largest out x in degree sits in a 2-cycle with 200 arcs
    out to sinks and 200 in from sources, and one arc into a 50-cycle: the
    first search settles the 2-cycle, the 50-cycle is found in a later
    round."""
    hub = ([0, 1], [1, 0])
    outs = (np.zeros(200), np.arange(300, 500))
    ins = (np.arange(500, 700), np.zeros(200))
    link = ([0], [100])
    a, b = _cat(hub, outs, ins, link, _cycle(np.arange(100, 150)))
    _check_directed_build(cc, 700, a, b)


def test_directed_build_chain_and_ties(cc):
    """Cycles of sizes 3..12 chained one way (one weak component, ten
    strong ones) next to separate 12-cycles: the largest size ties between
    parts and the one holding the smallest id wins; ids interleave so that
    the winner is not the first part found."""
    rng = np.random.default_rng(5)
    ids = rng.permutation(400)
    parts, at, heads = [], 0, []
    for size in range(3, 13):
        cyc = ids[at:at + size]
        at += size
        parts.append(_cycle(cyc))
        heads.append(cyc[0])
    parts += [(heads[:-1], heads[1:])]                 # chain A -> B -> ...
    for _ in range(4):                                  # separate 12-cycles
        parts.append(_cycle(ids[at:at + 12]))
        at += 12
    a, b = _cat(*parts)
    _check_directed_build(cc, 400, a, b)


def test_directed_build_acyclic_rejected(cc):
    """A directed acyclic graph has only one-node components: no graph to
    keep."""
    a, b = _cat((np.arange(0, 99), np.arange(1, 100)), (np.zeros(50), np.arange(50, 100)))
    with pytest.raises(cc.CCError):
        cc.cc_graph_from_edges(100, a, b, directed=True)


def test_directed_build_all_nodes(cc):
    n, s, d = synth.rmat_edges(11, 4, seed=21)
    _check_directed_build(cc, n, s, d, keep=False)


@pytest.mark.parametrize("n,k,seed", [(10, 3, 0), (1000, 64, 2), (5000, 1, 7),
                                      (3000, 2048, 5), (70000, 256, 11), (300, 300, 1)])
def test_sample_choose_matches_oracle(cc, n, k, seed):
    g, _ = cc.cc_graph_from_edges(*synth.path_edges(n))
    try:
        assert (cc.cc_sample_choose(g, k, seed) == orc.choose_sample(n, k, seed)).all()
    finally:
        cc.cc_graph_free(g)


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("k", [1, 5, 64, 100, 256, 300])
def test_estimate_parity(cc, name, k):
    n, s, d = GRAPHS[name]()
    g, old, og = both(cc, n, s, d)
    try:
        k = min(k, og.n)
        C = orc.choose_sample(og.n, k, 17 + k)
        for eps in [(1, 1), (1, 3), orc.default_eps(k)]:
            check_estimate(cc, g, og, C, eps)
    finally:
        cc.cc_graph_free(g)


def test_word_boundaries_and_large_k(cc):
    n, s, d = synth.rmat_edges(10, 8, seed=12)
    g, old, og = both(cc, n, s, d)
    try:
        for k in (63, 64, 65, 127, 128, 129, 511, 512, 513, 1024, 2048):
            C = orc.choose_sample(og.n, min(k, og.n), k)
            check_estimate(cc, g, og, C, (1, 2))
    finally:
        cc.cc_graph_free(g)


def test_full_sample_is_exact(cc):
    n, s, d = synth.grid_edges(12, 9)
    g, old, og = both(cc, n, s, d)
    try:
        C = orc.choose_sample(og.n, og.n, 3)
        r, _ = check_estimate(cc, g, og, C, (1, 2))
        S = orc.exact_S(og).astype(np.float64)
        for e in range(4):
            assert (r["s_hat"][e] == S).all()
    finally:
        cc.cc_graph_free(g)


def test_exact_all_pairs_config1(cc):
    """R-MAT scale 12, edge factor 8, seed 1, LCC: exact closeness of every
    node against the oracle's n BFS."""
    n, s, d = synth.rmat_edges(12, 8, seed=1)
    g, old, og = both(cc, n, s, d)
    try:
        c, S = cc.cc_exact(g)
        want = orc.exact_S(og)
        assert (S == want).all()
        assert_close(c, orc.exact_closeness(want), "exact closeness")
    finally:
        cc.cc_graph_free(g)


def test_estimate_config1(cc):
    """R-MAT scale 12 / edge factor 8 / seed 1, k = 64 (sample seed 2),
    eps = 1/8: every output."""
    n, s, d = synth.rmat_edges(12, 8, seed=1)
    g, old, og = both(cc, n, s, d)
    try:
        C = cc.cc_sample_choose(g, 64, 2)
        assert (C == orc.choose_sample(og.n, 64, 2)).all()
        check_estimate(cc, g, og, C, (1, 8))
        s_single, S_single = cc.cc_sampling_sums_single(g, C)
        want = orc.streaming_pass(og, C)
        assert (s_single == want["sum"]).all() and (S_single == want["S_samp"]).all()
    finally:
        cc.cc_graph_free(g)


def test_errors(cc):
    n, s, d = synth.path_edges(50)
    g, _ = cc.cc_graph_from_edges(n, s, d)
    try:
        with pytest.raises(cc.CCError) as e:
            cc.cc_estimate(g, [1, 1, 2])
        assert e.value.code == cc.CC_ERR_ARG
        with pytest.raises(cc.CCError):
            cc.cc_estimate(g, [0, 60])
        o = cc.cc_opts_default(2)
        o.eps_num, o.eps_den = 3, 2  # eps > 1
        with pytest.raises(cc.CCError):
            cc.cc_estimate(g, [0, 1], o)
    finally:
        cc.cc_graph_free(g)
    # two components kept: closeness undefined
    src = np.array([0, 1, 3, 4], np.uint32)
    dst = np.array([1, 2, 4, 5], np.uint32)
    g, _ = cc.cc_graph_from_edges(6, src, dst, keep_component=False)
    try:
        with pytest.raises(cc.CCError) as e:
            cc.cc_estimate(g, [0, 4])
        assert e.value.code == cc.CC_ERR_DISCONNECTED
    finally:
        cc.cc_graph_free(g)


def test_bounded_barrier_wait_reports_timeout(cc):
    assert cc.cc_selftest_barrier_timeout(50_000_000) == cc.CC_ERR_TIMEOUT


def test_repeatable(cc):
    n, s, d = synth.rmat_edges(11, 16, seed=21)
    g, _ = cc.cc_graph_from_edges(n, s, d)
    try:
        C = cc.cc_sample_choose(g, 200, 4)
        a = cc.cc_estimate(g, C)
        for _ in range(3):
            b = cc.cc_estimate(g, C)
            for key in a:
                assert (a[key] == b[key]).all(), key
    finally:
        cc.cc_graph_free(g)


@pytest.mark.parametrize("k", [100, 301])
def test_hub_row_at_the_end_of_the_csr(cc, k):
    """A hub whose row is the last of the CSR, with an arc count that is not
    a multiple of 4: its last 256-entry chunk ends inside the array's last
    16 bytes, so the bottom-up scan stages those entries by plain loads
    (k = 100: level 1 is bottom-up and the hub pulls from its leaves)."""
    n = 302
    s = np.arange(n - 1, dtype=np.uint32)
    d = np.full(n - 1, n - 1, np.uint32)
    g, _, og = both(cc, n, s, d)
    try:
        assert cc.cc_graph_info(g)[1] % 4 == 2
        C = orc.choose_sample(og.n, k, 3)
        check_estimate(cc, g, og, C, orc.default_eps(k))
    finally:
        cc.cc_graph_free(g)


def test_pinned_host_outputs(cc):
    """Pinned host output buffers get the same values as pageable ones, on
    every repeat (the repeats replay the captured graph)."""
    torch = pytest.importorskip("torch")
    n, s, d = synth.rmat_edges(12, 16, seed=7)
    g, _, og = both(cc, n, s, d)
    try:
        k = 200
        C = orc.choose_sample(og.n, k, 9)
        want = cc.cc_estimate(g, C)
        nn = og.n
        host = {"s_hat": torch.empty((4, nn), dtype=torch.float64, pin_memory=True),
                "closeness": torch.empty((4, nn), dtype=torch.float64, pin_memory=True),
                "pivot": torch.empty(nn, dtype=torch.int32, pin_memory=True),
                "delta": torch.empty(nn, dtype=torch.int32, pin_memory=True),
                "sum": torch.empty(nn, dtype=torch.int64, pin_memory=True),
                "hyb": torch.empty((nn, 6), dtype=torch.int64, pin_memory=True)}
        o = cc.cc_out()
        for e in range(4):
            o.s_hat[e] = host["s_hat"][e].data_ptr()
            o.closeness[e] = host["closeness"][e].data_ptr()
        o.pivot, o.delta = host["pivot"].data_ptr(), host["delta"].data_ptr()
        o.sample_sum, o.hyb_int = host["sum"].data_ptr(), host["hyb"].data_ptr()
        opts = cc.cc_opts_default(k)
        for rep in range(4):
            for t in host.values():
                t.zero_()
            cc.cc_estimate(g, C, opts, o)
            assert (host["s_hat"].numpy() == want["s_hat"]).all(), rep
            assert (host["closeness"].numpy() == want["closeness"]).all(), rep
            assert (host["pivot"].numpy() == want["pivot"]).all(), rep
            assert (host["delta"].numpy().view(np.uint32) == want["delta"]).all(), rep
            assert (host["sum"].numpy().view(np.uint64) == want["sum"]).all(), rep
            assert (host["hyb"].numpy().view(np.uint64) == want["hyb"]).all(), rep
        assert cc.cc_last_call_graph(g)
    finally:
        cc.cc_graph_free(g)


def test_repeated_estimate_replays_one_graph(cc):
    """A bit-packed estimate called again with the same arguments and device
    output buffers replays a captured CUDA graph from the third call on:
    every call equals the oracle, across a change of eps and back, a
    change of the direction switch, and with capture switched off."""
    torch = pytest.importorskip("torch")
    n, s, d = synth.rmat_edges(12, 8, seed=3)
    g, _, og = both(cc, n, s, d)
    try:
        k = 100
        C = orc.choose_sample(og.n, k, 5)
        dev = torch.device("cuda", 0)
        shat = torch.zeros((4, og.n), dtype=torch.float64, device=dev)
        clo = torch.zeros((4, og.n), dtype=torch.float64, device=dev)
        piv = torch.zeros(og.n, dtype=torch.int32, device=dev)
        dlt = torch.zeros(og.n, dtype=torch.int32, device=dev)
        o = cc.cc_out()
        for e in range(4):
            o.s_hat[e], o.closeness[e] = shat[e].data_ptr(), clo[e].data_ptr()
        o.pivot, o.delta = piv.data_ptr(), dlt.data_ptr()
        opts = cc.cc_opts_default(k)
        opts.device_outputs = 1
        e0 = orc.default_eps(k)
        want = {e0: orc.estimate(og, C, eps=e0), (1, 2): orc.estimate(og, C, eps=(1, 2))}
        replays = []
        plan = [e0] * 4 + [(1, 2)] * 4 + [e0] * 4
        for i, eps in enumerate(plan):
            if i == 10:
                cc.cc_set_tuning(g, 3)
            opts.eps_num, opts.eps_den = eps
            shat.zero_()
            clo.zero_()
            piv.zero_()
            dlt.zero_()
            cc.cc_estimate(g, C, opts, o)
            torch.cuda.synchronize()
            replays.append(cc.cc_last_call_graph(g))
            assert (piv.cpu().numpy() == want[eps]["pivot"]).all(), i
            assert (dlt.cpu().numpy().view(np.uint32) == want[eps]["delta"]).all(), i
            assert cc.cc_last_call_timing(g)[0] >= 1
            for e in range(4):
                assert_close(shat[e].cpu().numpy(), want[eps]["s_hat"][e], f"{i} s_hat[{e}]")
                assert_close(clo[e].cpu().numpy(), want[eps]["closeness"][e], f"{i} clo[{e}]")
        # arguments first seen run directly; their next call captures and
        # replays; a change of eps or of the direction switch (call 10)
        # starts over (the first call of all also sizes the buffers)
        assert replays[:4] == [False, False, True, True], replays
        assert replays[4] is False and replays[7] is True, replays
        assert replays[8] is False and replays[9] is True, replays
        assert replays[10] is False and replays[11] is True, replays
        cc.cc_set_param(g, cc.CC_PARAM_ESTIMATE_GRAPH, 0)
        for _ in range(3):
            shat.zero_()
            cc.cc_estimate(g, C, opts, o)
            torch.cuda.synchronize()
            assert not cc.cc_last_call_graph(g)
            assert_close(shat[3].cpu().numpy(), want[e0]["s_hat"][3], "no graph")
    finally:
        cc.cc_graph_free(g)


def check_chunked(cc, g, og, C, eps, roundtrip=False, hybrid=True):
    o = cc.cc_opts_default(len(C))
    o.eps_num, o.eps_den, o.want_hybrid, o.roundtrip = eps[0], eps[1], int(hybrid), int(roundtrip)
    r = cc.cc_estimate(g, C, o)
    want = orc.estimate(og, C, eps=eps, roundtrip=roundtrip)
    for key in ("pivot", "delta", "sum", "S_samp", "delta_cc"):
        assert (r[key] == want[key]).all(), key
    for e in range(4 if hybrid else 3):
        assert_close(r["s_hat"][e], want["s_hat"][e], f"s_hat[{e}]")
        assert_close(r["closeness"][e], want["closeness"][e], f"closeness[{e}]")
    if hybrid:
        assert (r["hyb"] == want["hyb"]).all()


WEIGHTED = {
    "ws_w": lambda: (*synth.watts_strogatz_edges(600, 6, 0.1, seed=5),
                     synth.random_weights(1800, 1, 40, seed=6)),
    "rmat_w": lambda: (*synth.rmat_edges(9, 6, seed=7),
                       synth.random_weights(6 * 512, 1, 1000, seed=8)),
    "grid_w": lambda: (*synth.grid_edges(30, 20),
                       synth.random_weights(29 * 20 + 30 * 19, 1, 3, seed=9)),
}


@pytest.mark.parametrize("name", sorted(WEIGHTED))
@pytest.mark.parametrize("k", [1, 31, 32, 33, 64, 100])
def test_weighted_estimate_parity(cc, name, k):
    n, s, d, w = WEIGHTED[name]()
    g, old, og = both(cc, n, s, d, w)
    try:
        k = min(k, og.n)
        C = orc.choose_sample(og.n, k, 5 + k)
        for eps in [(1, 1), (1, 4), orc.default_eps(k)]:
            check_chunked(cc, g, og, C, eps)
    finally:
        cc.cc_graph_free(g)


def test_rgg_road_like_weights(cc):
    n, s, d, length = synth.rgg_edges(4000, 0.03, seed=3)
    w = synth.edge_lengths_to_weights(length, 1000.0)
    g, old, og = both(cc, n, s, d, w)
    try:
        C = orc.choose_sample(og.n, 64, 2)
        check_chunked(cc, g, og, C, (1, 8))
        c, S = cc.cc_exact(g)
        assert (S == orc.exact_S(og)).all()
    finally:
        cc.cc_graph_free(g)


DIRECTED = {
    "rmat_d": lambda: (*synth.rmat_edges(9, 8, seed=11), None),
    "rmat_dw": lambda: (*synth.rmat_edges(8, 8, seed=12),
                        synth.random_weights(8 * 256, 1, 9, seed=13)),
}


@pytest.mark.parametrize("name", sorted(DIRECTED))
@pytest.mark.parametrize("k", [1, 32, 50])
def test_roundtrip_estimate_parity(cc, name, k):
    n, s, d, w = DIRECTED[name]()
    g, old, og = both(cc, n, s, d, w, directed=True)
    try:
        k = min(k, og.n)
        C = orc.choose_sample(og.n, k, 3 + k)
        for eps in [(1, 1), (1, 3)]:
            check_chunked(cc, g, og, C, eps, roundtrip=True)
        with pytest.raises(cc.CCError):  # directed graphs need round trips
            cc.cc_estimate(g, C)
    finally:
        cc.cc_graph_free(g)


def test_exact_weighted_and_roundtrip(cc):
    n, s, d, w = WEIGHTED["ws_w"]()
    g, old, og = both(cc, n, s, d, w)
    try:
        c, S = cc.cc_exact(g)
        want = orc.exact_S(og)
        assert (S == want).all()
        assert_close(c, orc.exact_closeness(want), "exact weighted closeness")
    finally:
        cc.cc_graph_free(g)
    n, s, d, w = DIRECTED["rmat_d"]()
    g, old, og = both(cc, n, s, d, w, directed=True)
    try:
        c, S = cc.cc_exact(g)
        assert (S == orc.exact_S(og, roundtrip=True)).all()
    finally:
        cc.cc_graph_free(g)


ONE_PASS = {
    "grid": lambda: synth.grid_edges(61, 47),
    "ws": lambda: synth.watts_strogatz_edges(3000, 6, 0.02, seed=9),
    "rmat": lambda: synth.rmat_edges(11, 8, seed=5),
    "path": lambda: synth.path_edges(700),
}


@pytest.mark.parametrize("name", sorted(ONE_PASS))
@pytest.mark.parametrize("k", [3, 64, 100, 256])
def test_hybrid_in_first_pass(cc, name, k):
    """The hybrid classified on arrival (one traversal, deferred bits
    resolved after it) equals the oracle and the two-pass form, for eps
    down to 1/sqrt(k) and up to 1; long paths with few sources overflow the
    byte band and fall back to the second pass, still exact."""
    n, s, d = ONE_PASS[name]()
    g, old, og = both(cc, n, s, d)
    try:
        k = min(k, og.n)
        C = orc.choose_sample(og.n, k, 11 + k)
        for eps in [(1, 1), (1, 2), (2, 7), orc.default_eps(k)]:
            cc.cc_set_param(g, cc.CC_PARAM_HYBRID_ONE_PASS, 1)
            r1, want = check_estimate(cc, g, og, C, eps)
            cc.cc_set_param(g, cc.CC_PARAM_HYBRID_ONE_PASS, 0)
            o = cc.cc_opts_default(k)
            o.eps_num, o.eps_den = eps
            r2 = cc.cc_estimate(g, C, o)
            for key in ("hyb", "sum", "pivot", "delta"):
                assert (r1[key] == r2[key]).all(), (eps, key)
            assert (r1["s_hat"] == r2["s_hat"]).all(), eps
    finally:
        cc.cc_graph_free(g)


def test_hybrid_in_first_pass_runs_one_traversal(cc):
    """On a grid, where some L(v) misses sampled nodes, the hybrid needs
    one traversal launch instead of two."""
    n, s, d = synth.grid_edges(120, 90)
    g, _ = cc.cc_graph_from_edges(n, s, d)
    try:
        C = cc.cc_sample_choose(g, 128, 4)
        cc.cc_estimate(g, C)
        assert cc.cc_last_call_timing(g)[0] == 1
        cc.cc_set_param(g, cc.CC_PARAM_HYBRID_ONE_PASS, 0)
        cc.cc_estimate(g, C)
        assert cc.cc_last_call_timing(g)[0] == 2
    finally:
        cc.cc_graph_free(g)
