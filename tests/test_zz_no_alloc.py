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


def test_no_alloc_refuses_sizes_beyond_its_array(cc):
    import torch
    n = 3_000_000  # 4 * n * 8 bytes of words alone exceed the fixed array
    dummy = torch.zeros(8, dtype=torch.int64, device="cuda")
    rc = cc.cc_sampling_pivots_noalloc(n, dummy.data_ptr(), dummy.data_ptr(), [0, 1],
                                       dummy.data_ptr(), dummy.data_ptr(),
                                       dummy.data_ptr(), dummy.data_ptr())
    assert rc == cc.CC_ERR_TOO_LARGE
