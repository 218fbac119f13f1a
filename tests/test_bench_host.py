"""Host-side pieces of bench.py: the multi-core CPU baseline's merge of
per-thread streaming passes gives the single-thread pass's outputs."""
import numpy as np
import pytest

import synth
from oracle import oracle as orc


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_threaded_streaming_pass_equals_single(threads):
    import bench
    n, s, d = synth.rmat_edges(10, 8, seed=2)
    og = orc.csr_from_edges(n, s, d)
    for k in (5, 40):
        C = orc.choose_sample(og.n, k, 3)
        want = orc.streaming_pass(og, C)
        got = bench.streaming_pass_threads(og, C, threads)
        for key in ("sum", "pivot", "delta", "S_samp"):
            assert (got[key] == want[key]).all(), (threads, k, key)


def test_host_cpu_reports_cores():
    import bench
    cores, model = bench.host_cpu()
    assert cores >= 1 and isinstance(model, str) and model
