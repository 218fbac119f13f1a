"""Batched persistent launch: every graph's results equal the single-graph
path's bit for bit and the oracle's, twice in a row, with and without
autotuning."""
import numpy as np
import pytest

import synth
from oracle import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    from paper_1409_0035_gb300 import build
    build.build()
    import paper_1409_0035_gb300 as m
    return m


def mixed_batch():
    gens = [synth.rmat_edges(9, 8, seed=1), synth.rmat_edges(11, 16, seed=2),
            synth.grid_edges(40, 25), synth.grid_edges(9, 7),
            synth.watts_strogatz_edges(1500, 10, 0.05, seed=3),
            synth.rmat_edges(8, 12, seed=4), synth.path_edges(400),
            synth.star_edges(600), synth.rmat_edges(12, 8, seed=5),
            synth.watts_strogatz_edges(4096, 10, 0.05, seed=6)]
    ks = [16, 64, 256, 20, 512, 3, 64, 100, 256, 64]
    return gens, ks


@pytest.mark.parametrize("autotune", [True, False])
def test_batch_matches_single(cc, autotune):
    gens, ks = mixed_batch()
    handles, samples, olds, ns = [], [], [], []
    try:
        for (n, s, d), k in zip(gens, ks):
            g, old = cc.cc_graph_from_edges(n, s, d)
            handles.append(g)
            nn = cc.cc_graph_info(g)[0]
            ns.append(nn)
            samples.append(cc.cc_sample_choose(g, min(k, nn), 7 + k))
        b = cc.cc_batch_create(handles, samples, autotune=autotune)
        try:
            info = cc.cc_batch_info(b)
            assert 1 <= info["teams"] <= 64
            for rep in range(2):
                cc.cc_batch_run(b)
                for i, g in enumerate(handles):
                    got = cc.cc_batch_result(b, i, ns[i], len(samples[i]))
                    want = cc.cc_estimate(g, samples[i])
                    for key in want:
                        assert (got[key] == want[key]).all(), (i, key)
            info = cc.cc_batch_info(b)
            assert info["last_ms"] > 0
        finally:
            cc.cc_batch_free(b)
        # every graph of the batch against the oracle (the batch equals the
        # single-graph call, checked above)
        for i, (n, s, d) in enumerate(gens):
            og = orc.csr_from_edges(n, s, d)
            k = len(samples[i])
            want = orc.estimate(og, samples[i], eps=orc.default_eps(k))
            got = cc.cc_estimate(handles[i], samples[i])
            for key in ("pivot", "delta", "sum", "S_samp", "delta_cc", "hyb"):
                assert (got[key] == want[key]).all(), (i, key)
            assert np.allclose(got["s_hat"], want["s_hat"], rtol=1e-12, atol=0), i
            assert np.allclose(got["closeness"], want["closeness"], rtol=1e-12, atol=0), i
    finally:
        for g in handles:
            cc.cc_graph_free(g)


def test_autotune_cache(cc, tmp_path):
    """The first autotuned batch times its graphs and writes one cache line
    per graph; a second batch of the same graphs takes every graph's
    tuning from the file (same direction switch) and still equals the
    single-graph calls."""
    gens, ks = mixed_batch()
    path = tmp_path / "tune.jsonl"
    handles, samples, ns = [], [], []
    try:
        for (n, s, d), k in zip(gens, ks):
            g, _ = cc.cc_graph_from_edges(n, s, d)
            handles.append(g)
            nn = cc.cc_graph_info(g)[0]
            ns.append(nn)
            samples.append(cc.cc_sample_choose(g, min(k, nn), 7 + k))
        cc.cc_batch_tune_cache(path)
        try:
            b1 = cc.cc_batch_create(handles, samples, autotune=True)
            p1 = [cc.cc_batch_plan(b1, i) for i in range(len(handles))]
            cc.cc_batch_free(b1)
            lines = path.read_text().splitlines()
            assert len(lines) == len(handles)
            assert not any(p["from_cache"] for p in p1)
            b2 = cc.cc_batch_create(handles, samples, autotune=True)
            try:
                p2 = [cc.cc_batch_plan(b2, i) for i in range(len(handles))]
                assert all(p["from_cache"] for p in p2)
                assert [p["alpha"] for p in p1] == [p["alpha"] for p in p2]
                assert len(path.read_text().splitlines()) == len(handles)
                cc.cc_batch_run(b2)
                for i, g in enumerate(handles):
                    got = cc.cc_batch_result(b2, i, ns[i], len(samples[i]))
                    want = cc.cc_estimate(g, samples[i])
                    for key in want:
                        assert (got[key] == want[key]).all(), (i, key)
            finally:
                cc.cc_batch_free(b2)
        finally:
            cc.cc_batch_tune_cache(None)
    finally:
        for g in handles:
            cc.cc_graph_free(g)
