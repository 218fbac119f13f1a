"""C-ABI library loads and exports every symbol include/cc.h declares; host
logic that needs no GPU.  CPU only (no compute call)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import shutil
    if shutil.which("nvcc") is None:
        pytest.skip("nvcc not available")
    from paper_1409_0035_gb300 import build
    build.build()
    import paper_1409_0035_gb300 as cc
    return cc.lib()


def declared_functions():
    names = []
    for hdr in ("cc.h",):
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(cc_\w+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    import paper_1409_0035_gb300 as cc
    decl = declared_functions()
    assert len(decl) >= 13
    for name in decl:
        assert hasattr(lib, name), name
    assert set(cc.EXPORTS) <= set(decl)
    nm = subprocess.run(["nm", "-D", "--defined-only", cc.LIB_PATH],
                        capture_output=True, text=True).stdout
    for name in decl:
        assert re.search(rf"\bT {name}\b", nm), name


def test_strerror_and_defaults_are_host_only(lib):
    import paper_1409_0035_gb300 as cc
    assert cc.cc_strerror(cc.CC_ERR_DISCONNECTED).startswith("graph not")
    assert cc.cc_strerror(12345) == "unknown error"
    o = cc.cc_opts_default(256)
    assert (o.eps_num, o.eps_den, o.want_hybrid, o.roundtrip) == (1, 16, 1, 0)
    o = cc.cc_opts_default(100)
    assert (o.eps_num, o.eps_den) == (1, 10)  # section 7: eps = sqrt(1/k) = 0.1


def test_graph_build_without_device_reports_no_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    import paper_1409_0035_gb300 as cc
    with pytest.raises(cc.CCError) as e:
        cc.cc_graph_from_edges(3, np.array([0, 1]), np.array([1, 2]))
    assert e.value.code == cc.CC_ERR_NO_DEVICE


def test_binding_constants_match_the_header():
    """Every CC_* constant the binding defines equals the header's #define
    of the same name (error codes, estimator indices, parameters, limits)."""
    import paper_1409_0035_gb300 as cc
    text = open(os.path.join(ROOT, "include", "cc.h")).read()
    defines = {m.group(1): int(m.group(2))
               for m in re.finditer(r"#define\s+(CC_\w+)\s+\(?(-?\d+)\)?", text)}
    names = [n for n in dir(cc) if n.startswith("CC_") and isinstance(getattr(cc, n), int)]
    assert len(names) >= 20
    for n in names:
        assert n in defines, n
        assert getattr(cc, n) == defines[n], n
