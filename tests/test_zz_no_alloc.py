"""The allocation-free entry point against the regular one.

cc_sampling_pivots_noalloc serves callers that cannot allocate device memory
(a framework's memory pool owns the device, or a budget forbids allocations
mid-run): it keeps its working memory in a fixed device array inside the
library.  Here the caller-side buffers come from torch; the call itself must
reproduce cc_estimate's first-pass outputs exactly, twice in a row (the
second call reuses the array the first one left dirty), and refuse a size
beyond its fixed array.  This file runs last so that a failure here comes
after every other test has run.
"""
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


def _run(cc, torch, n, rp, col, C):
    dev = torch.device("cuda", 0)
    d_rp = torch.from_numpy(rp).to(dev)
    d_col = torch.from_numpy(col).to(dev)
    out = dict(sum=torch.zeros(n, dtype=torch.int64, device=dev),
               pivot=torch.zeros(n, dtype=torch.int32, device=dev),
               delta=torch.zeros(n, dtype=torch.int32, device=dev),
               S=torch.zeros(len(C), dtype=torch.int64, device=dev))
    rc = cc.cc_sampling_pivots_noalloc(
        n, d_rp.data_ptr(), d_col.data_ptr(), C, out["sum"].data_ptr(),
        out["pivot"].data_ptr(), out["delta"].data_ptr(), out["S"].data_ptr(),
        torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return rc, {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("scale,k,seed", [(12, 64, 2), (13, 200, 5)])
def test_no_alloc_matches_estimate_twice(cc, scale, k, seed):
    import torch
    n0, s, d = synth.rmat_edges(scale, 8, seed=1)
    g, _ = cc.cc_graph_from_edges(n0, s, d)
    try:
        n = cc.cc_graph_info(g)[0]
        rp, col, _ = cc.cc_graph_copy_csr(g)
        C = cc.cc_sample_choose(g, k, seed)
        o = cc.cc_opts_default(k)
        o.want_hybrid = 0
        want = cc.cc_estimate(g, C, o)
        for _ in range(2):
            rc, got = _run(cc, torch, n, rp, col, C)
            assert rc == cc.CC_OK, cc.cc_strerror(rc)
            assert (got["sum"].view(np.uint64) == want["sum"]).all()
            assert (got["pivot"] == want["pivot"]).all()
            assert (got["delta"].view(np.uint32) == want["delta"]).all()
            assert (got["S"].view(np.uint64) == want["S_samp"]).all()
    finally:
        cc.cc_graph_free(g)
    # and against the oracle's running-state pass on its own CSR of the graph
    og = orc.csr_from_edges(n0, s, d)
    assert (og.row_ptr == rp).all() and (og.col == col).all()
    ref = orc.streaming_pass(og, C)
    assert (got["sum"].view(np.uint64) == ref["sum"]).all()
    assert (got["pivot"] == ref["pivot"]).all()
    assert (got["delta"].view(np.uint32) == ref["delta"]).all()
    assert (got["S"].view(np.uint64) == ref["S_samp"]).all()


def test_no_alloc_level_limit_then_normal_call(cc):
    """A path of 2100 nodes sampled at one end needs 2099 levels, more than
    the fixed distance histogram holds: the call reports CC_ERR_TOO_LARGE
    (after the pass), and the array it left behind does not disturb the
    next, normal call."""
    import torch
    n, s, d = synth.path_edges(2100)
    og = orc.csr_from_edges(n, s, d)
    rc, _ = _run(cc, torch, og.n, og.row_ptr, og.col, np.array([0, 1], np.int32))
    assert rc == cc.CC_ERR_TOO_LARGE
    n0, s, d = synth.rmat_edges(11, 8, seed=4)
    og = orc.csr_from_edges(n0, s, d)
    C = orc.choose_sample(og.n, 100, 9)
    rc, got = _run(cc, torch, og.n, og.row_ptr, og.col, C)
    assert rc == cc.CC_OK, cc.cc_strerror(rc)
    ref = orc.streaming_pass(og, C)
    assert (got["sum"].view(np.uint64) == ref["sum"]).all()
    assert (got["pivot"] == ref["pivot"]).all()
    assert (got["delta"].view(np.uint32) == ref["delta"]).all()
    assert (got["S"].view(np.uint64) == ref["S_samp"]).all()


def test_no_alloc_rejects_one_way_csr(cc):
    """A directed cycle (every arc one way) has in-degree 1 and out-degree 1
    everywhere -- passes the degree check -- so a one-way path is used: its
    first node has an arc out and none in."""
    import torch
    n = 50
    rp = np.concatenate([np.arange(n, dtype=np.int64), [n - 1]])
    col = np.arange(1, n, dtype=np.int32)
    rc, _ = _run(cc, torch, n, rp, col, np.array([0, 7], np.int32))
    assert rc == cc.CC_ERR_GRAPH


def test_no_alloc_refuses_sizes_beyond_its_array(cc):
    import torch
    n = 3_000_000  # 4 * n * 8 bytes of words alone exceed the fixed array
    dummy = torch.zeros(8, dtype=torch.int64, device="cuda")
    rc = cc.cc_sampling_pivots_noalloc(n, dummy.data_ptr(), dummy.data_ptr(), [0, 1],
                                       dummy.data_ptr(), dummy.data_ptr(),
                                       dummy.data_ptr(), dummy.data_ptr())
    assert rc == cc.CC_ERR_TOO_LARGE
