"""Thin Python binding of libcc_gb300.so (the C ABI in include/cc.h).

Every cc_* function here marshals arguments and calls the C entry point of
the same name; all computation runs in the library's sm_103a kernels.  The
library must be built (``paper_1409_0035_gb300.build.build()``); importing
fails loudly when it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcc_gb300.so")

CC_OK = 0
CC_ERR_ARG = -1
CC_ERR_GRAPH = -2
CC_ERR_DISCONNECTED = -3
CC_ERR_OOM = -4
CC_ERR_TIMEOUT = -5
CC_ERR_CUDA = -6
CC_ERR_TOO_LARGE = -7
CC_ERR_NO_DEVICE = -8
CC_MAX_K = 2048
# estimators (index of cc_out.s_hat / closeness and of the result arrays)
CC_EST_SAMPLING, CC_EST_PIVOTING, CC_EST_PIVOT_UPPER, CC_EST_HYBRID = 0, 1, 2, 3
CC_NUM_EST = 4
EST_NAMES = ("sampling", "pivoting", "pivot_upper", "hybrid")

# Every symbol include/cc.h declares.
EXPORTS = (
    "cc_graph_from_edges", "cc_graph_load_csr", "cc_graph_free", "cc_graph_info",
    "cc_graph_copy_csr", "cc_sample_choose", "cc_opts_default", "cc_estimate",
    "cc_exact", "cc_sampling_sums_single", "cc_last_pass_stats",
    "cc_last_call_timing", "cc_last_call_graph", "cc_sampling_pivots_noalloc",
    "cc_last_pass_trace",
    "cc_set_tuning", "cc_set_param", "cc_batch_create", "cc_batch_run", "cc_batch_result",
    "cc_batch_info", "cc_batch_plan", "cc_batch_tune_cache", "cc_batch_free", "cc_server_create", "cc_server_submit",
    "cc_server_wait", "cc_server_result", "cc_server_stats", "cc_server_cache_stats",
    "cc_server_free",
    "cc_selftest_barrier_timeout", "cc_strerror", "cc_last_pass_phases",
    "cc_estimate_adaptive", "cc_graph_set_node_weights", "cc_sample_varopt",
    "cc_estimate_node_weighted", "cc_reach_estimate",
)

PHASES = ("init", "td_queue", "td_push", "td_final", "bu_rebuild", "bu_light",
          "bu_medium", "bu_heavy", "bu_final", "barrier")


class CCError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {cc_strerror(code)} ({code})")
        self.code = code


class cc_opts(ctypes.Structure):
    _fields_ = [("eps_num", ctypes.c_uint32), ("eps_den", ctypes.c_uint32),
                ("want_hybrid", ctypes.c_int32), ("roundtrip", ctypes.c_int32),
                ("device_outputs", ctypes.c_int32), ("stream", ctypes.c_void_p)]


class cc_out(ctypes.Structure):
    _fields_ = [("s_hat", ctypes.c_void_p * CC_NUM_EST),
                ("closeness", ctypes.c_void_p * CC_NUM_EST),
                ("pivot", ctypes.c_void_p), ("delta", ctypes.c_void_p),
                ("sample_sum", ctypes.c_void_p), ("hyb_int", ctypes.c_void_p),
                ("S_sampled", ctypes.c_void_p), ("delta_cc", ctypes.c_void_p),
                ("sq_err", ctypes.c_void_p)]


class cc_wout(ctypes.Structure):
    _fields_ = [("s_hat", ctypes.c_void_p * 2), ("closeness", ctypes.c_void_p * 2),
                ("S_sampled", ctypes.c_void_p)]


_lib = None


def lib():
    """Load libcc_gb300.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run "
                              "paper_1409_0035_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        P, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
        c_int = ctypes.c_int
        L.cc_graph_from_edges.argtypes = [i64, i64, P, P, P, c_int, c_int, P, P]
        L.cc_graph_load_csr.argtypes = [i64, P, P, P, c_int, c_int, P, P]
        L.cc_graph_free.argtypes = [P]
        L.cc_graph_info.argtypes = [P, P, P, P, P]
        L.cc_graph_copy_csr.argtypes = [P, c_int, P, P, P]
        L.cc_sample_choose.argtypes = [P, i32, u64, P]
        L.cc_opts_default.argtypes = [P, i32]
        L.cc_opts_default.restype = None
        L.cc_estimate.argtypes = [P, P, i32, P, P]
        L.cc_estimate_adaptive.argtypes = [P, P, i32, P, i32, P, P, P, P, P, P]
        L.cc_exact.argtypes = [P, P, P]
        L.cc_graph_set_node_weights.argtypes = [P, P]
        L.cc_sample_varopt.argtypes = [P, i32, u64, P, P]
        L.cc_estimate_node_weighted.argtypes = [P, P, i32, P, P, P]
        L.cc_reach_estimate.argtypes = [P, i32, u64, i32, P, P, P, P, P, P]
        L.cc_sampling_sums_single.argtypes = [P, P, i32, P, P]
        L.cc_last_pass_stats.argtypes = [P, P, P, P, P, P]
        L.cc_last_pass_phases.argtypes = [P, P]
        L.cc_last_call_timing.argtypes = [P, P, P, P, P]
        L.cc_last_call_graph.argtypes = [P, P]
        L.cc_last_pass_trace.argtypes = [P, i32, P, P, P, P, P]
        L.cc_set_tuning.argtypes = [P, i32]
        L.cc_set_param.argtypes = [P, i32, i32]
        L.cc_batch_create.argtypes = [i32, P, P, P, P, P, i32, P]
        L.cc_batch_run.argtypes = [P, P]
        L.cc_batch_result.argtypes = [P, i32, P, i32]
        L.cc_batch_info.argtypes = [P, P, P, P, P]
        L.cc_batch_plan.argtypes = [P, i32, P, P, P, P, P, P, P]
        L.cc_batch_tune_cache.argtypes = [ctypes.c_char_p]
        L.cc_batch_free.argtypes = [P]
        L.cc_server_create.argtypes = [i32, P, i32, u64, P]
        L.cc_server_submit.argtypes = [P, i32, i32, i32, u64, ctypes.c_uint32, ctypes.c_uint32, P]
        L.cc_server_wait.argtypes = [P, i64, i32]
        L.cc_server_result.argtypes = [P, i64, P, P, P, P, P, P]
        L.cc_server_stats.argtypes = [P, P, P, P, P, P]
        L.cc_server_cache_stats.argtypes = [P, P, P, P, P]
        L.cc_server_free.argtypes = [P]
        L.cc_sampling_pivots_noalloc.argtypes = [i64, P, P, P, i32, P, P, P, P, P]
        L.cc_selftest_barrier_timeout.argtypes = [u64]
        L.cc_strerror.argtypes = [c_int]
        L.cc_strerror.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    return a.ctypes.data_as(ctypes.c_void_p)


def _chk(rc, what):
    if rc != CC_OK:
        raise CCError(rc, what)


def cc_strerror(code: int) -> str:
    return lib().cc_strerror(int(code)).decode()


# ---------------------------------------------------------------- graphs

def cc_graph_from_edges(n, src, dst, w=None, directed=False, keep_component=True):
    """Returns (handle, old_id) -- see include/cc.h."""
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    ww = None if w is None else np.ascontiguousarray(w, dtype=np.uint32)
    h = ctypes.c_void_p()
    old = np.empty(int(n), dtype=np.int32)
    _chk(lib().cc_graph_from_edges(int(n), src.size, _p(src), _p(dst), _p(ww),
                                   int(directed), int(keep_component),
                                   ctypes.byref(h), _p(old)), "cc_graph_from_edges")
    nn = cc_graph_info(h.value)[0]
    return h.value, old[:nn].copy()


def cc_graph_load_csr(n, row_ptr, col, w=None, directed=False, keep_component=True):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    ww = None if w is None else np.ascontiguousarray(w, dtype=np.uint32)
    h = ctypes.c_void_p()
    old = np.empty(int(n), dtype=np.int32)
    _chk(lib().cc_graph_load_csr(int(n), _p(rp), _p(cl), _p(ww), int(directed),
                                 int(keep_component), ctypes.byref(h), _p(old)),
         "cc_graph_load_csr")
    nn = cc_graph_info(h.value)[0]
    return h.value, old[:nn].copy()


def cc_graph_free(g):
    _chk(lib().cc_graph_free(g), "cc_graph_free")


def cc_graph_info(g):
    """(n, arcs, directed, weighted)."""
    n, a = ctypes.c_int64(), ctypes.c_int64()
    d, w = ctypes.c_int(), ctypes.c_int()
    _chk(lib().cc_graph_info(g, ctypes.byref(n), ctypes.byref(a), ctypes.byref(d),
                             ctypes.byref(w)), "cc_graph_info")
    return n.value, a.value, bool(d.value), bool(w.value)


def cc_graph_copy_csr(g, reverse=False):
    n, arcs, _, weighted = cc_graph_info(g)
    rp = np.empty(n + 1, np.int64)
    col = np.empty(arcs, np.int32)
    w = np.empty(arcs, np.uint32) if weighted else None
    _chk(lib().cc_graph_copy_csr(g, int(reverse), _p(rp), _p(col), _p(w)),
         "cc_graph_copy_csr")
    return rp, col, w


# ---------------------------------------------------------------- estimation

def cc_sample_choose(g, k, seed):
    out = np.empty(int(k), np.int32)
    _chk(lib().cc_sample_choose(g, int(k), ctypes.c_uint64(seed & (2**64 - 1)),
                                _p(out)), "cc_sample_choose")
    return out


def cc_opts_default(k):
    o = cc_opts()
    lib().cc_opts_default(ctypes.byref(o), int(k))
    return o


def cc_estimate(g, sample, opts=None, out=None, want_sqerr=False):
    """Low-level call: `out` is a filled cc_out (host or device pointers per
    opts.device_outputs).  Without `out`, allocates host numpy outputs and
    returns them as a dict (with "sq_err", the hybrid's error estimate, when
    want_sqerr)."""
    sample = np.ascontiguousarray(sample, dtype=np.int32)
    k = sample.size
    if opts is None:
        opts = cc_opts_default(k)
    if out is not None:
        _chk(lib().cc_estimate(g, _p(sample), k, ctypes.byref(opts), ctypes.byref(out)),
             "cc_estimate")
        return out
    n = cc_graph_info(g)[0]
    res = dict(s_hat=np.zeros((CC_NUM_EST, n)), closeness=np.zeros((CC_NUM_EST, n)),
               pivot=np.empty(n, np.int32), delta=np.empty(n, np.uint32),
               sum=np.empty(n, np.uint64), hyb=np.zeros((n, 6), np.uint64),
               S_samp=np.empty(k, np.uint64), delta_cc=np.empty((k, k), np.uint32))
    o = cc_out()
    for e in range(CC_NUM_EST):
        o.s_hat[e] = _p(res["s_hat"][e])
        o.closeness[e] = _p(res["closeness"][e])
    o.pivot, o.delta = _p(res["pivot"]), _p(res["delta"])
    o.sample_sum, o.hyb_int = _p(res["sum"]), _p(res["hyb"])
    o.S_sampled, o.delta_cc = _p(res["S_samp"]), _p(res["delta_cc"])
    if want_sqerr:
        res["sq_err"] = np.empty(n, np.float64)
        o.sq_err = _p(res["sq_err"])
    _chk(lib().cc_estimate(g, _p(sample), k, ctypes.byref(opts), ctypes.byref(o)),
         "cc_estimate")
    return res


ADAPTIVE_EPS = ((1, 1000), (1, 40), (1, 20), (1, 10), (1, 5), (1, 2), (99, 100))


def cc_estimate_adaptive(g, sample, opts=None, eps_list=None):
    """Adaptive hybrid: per node the eq. (4) estimate of the eps (from
    eps_list, default the paper's seven values) with the smallest SqErrEst.
    Returns a dict of host arrays s_hat, closeness, sq_err, choice."""
    sample = np.ascontiguousarray(sample, dtype=np.int32)
    k = sample.size
    if opts is None:
        opts = cc_opts_default(k)
    n = cc_graph_info(g)[0]
    res = dict(s_hat=np.empty(n), closeness=np.empty(n), sq_err=np.empty(n),
               choice=np.empty(n, np.int32))
    if eps_list is None:
        ne, a, b = 0, None, None
    else:
        ne = len(eps_list)
        a = np.ascontiguousarray([e[0] for e in eps_list], np.uint32)
        b = np.ascontiguousarray([e[1] for e in eps_list], np.uint32)
    _chk(lib().cc_estimate_adaptive(g, _p(sample), k, ctypes.byref(opts), ne, _p(a), _p(b),
                                    _p(res["s_hat"]), _p(res["closeness"]),
                                    _p(res["sq_err"]), _p(res["choice"])),
         "cc_estimate_adaptive")
    return res


def cc_graph_set_node_weights(g, beta):
    """Attach node weights beta (uint32[n], the graph's numbering; None
    detaches) for the node-weighted estimates of section 5."""
    if beta is None:
        _chk(lib().cc_graph_set_node_weights(g, None), "cc_graph_set_node_weights")
        return
    b = np.ascontiguousarray(beta, dtype=np.uint32)
    if b.size != cc_graph_info(g)[0]:
        raise ValueError("need one weight per node")
    _chk(lib().cc_graph_set_node_weights(g, _p(b)), "cc_graph_set_node_weights")


def cc_sample_varopt(g, k, seed):
    """Weighted sample of exactly k nodes (section 5): returns (sample int32[k],
    tau as the fraction (numerator, denominator))."""
    out = np.empty(int(k), np.int32)
    tau = np.zeros(2, np.uint64)
    _chk(lib().cc_sample_varopt(g, int(k), ctypes.c_uint64(seed & (2**64 - 1)), _p(out),
                                _p(tau)), "cc_sample_varopt")
    return out, (int(tau[0]), int(tau[1]))


def cc_estimate_node_weighted(g, sample, tau, opts=None, out=None):
    """Node-weighted estimates (section 5) from a weighted sample and its tau.
    With `out` (a filled cc_wout) the call writes there; otherwise returns
    a dict of host arrays s_hat (2 x n: sampling, hybrid), closeness (2 x n)
    and S_sampled (k)."""
    sample = np.ascontiguousarray(sample, dtype=np.int32)
    k = sample.size
    t = np.ascontiguousarray([int(tau[0]), int(tau[1])], dtype=np.uint64)
    if opts is None:
        opts = cc_opts_default(k)
    if out is not None:
        _chk(lib().cc_estimate_node_weighted(g, _p(sample), k, _p(t), ctypes.byref(opts),
                                             ctypes.byref(out)), "cc_estimate_node_weighted")
        return out
    n = cc_graph_info(g)[0]
    res = dict(s_hat=np.zeros((2, n)), closeness=np.zeros((2, n)),
               S_sampled=np.empty(k, np.uint64))
    o = cc_wout()
    for e in range(2):
        o.s_hat[e] = _p(res["s_hat"][e])
        o.closeness[e] = _p(res["closeness"][e])
    o.S_sampled = _p(res["S_sampled"])
    _chk(lib().cc_estimate_node_weighted(g, _p(sample), k, _p(t), ctypes.byref(opts),
                                         ctypes.byref(o)), "cc_estimate_node_weighted")
    return res


def cc_reach_estimate(g, k, seed, inbound=False, stream=None):
    """Outbound (inbound) estimates of section 6.2: dict of host arrays avg
    (average distance to each node's bottom-k reachability sample), R_hat
    (size of the reachability set), count, distsum, T."""
    n = cc_graph_info(g)[0]
    res = dict(avg=np.empty(n), R_hat=np.empty(n), count=np.empty(n, np.int32),
               distsum=np.empty(n, np.uint64), T=np.empty(n, np.int64))
    _chk(lib().cc_reach_estimate(g, int(k), ctypes.c_uint64(seed & (2**64 - 1)),
                                 int(bool(inbound)), stream, _p(res["avg"]), _p(res["R_hat"]),
                                 _p(res["count"]), _p(res["distsum"]), _p(res["T"])),
         "cc_reach_estimate")
    return res


def cc_exact(g):
    """(closeness, S) for every node."""
    n = cc_graph_info(g)[0]
    c = np.empty(n, np.float64)
    S = np.empty(n, np.uint64)
    _chk(lib().cc_exact(g, _p(c), _p(S)), "cc_exact")
    return c, S


def cc_sampling_sums_single(g, sample):
    sample = np.ascontiguousarray(sample, dtype=np.int32)
    n = cc_graph_info(g)[0]
    s = np.empty(n, np.uint64)
    S = np.empty(sample.size, np.uint64)
    _chk(lib().cc_sampling_sums_single(g, _p(sample), sample.size, _p(s), _p(S)),
         "cc_sampling_sums_single")
    return s, S


def cc_last_pass_stats(g):
    vals = [ctypes.c_int64() for _ in range(5)]
    _chk(lib().cc_last_pass_stats(g, *[ctypes.byref(v) for v in vals]),
         "cc_last_pass_stats")
    return dict(zip(("levels", "td_levels", "bu_levels", "edges", "words"),
                    [v.value for v in vals]))


def cc_last_pass_phases(g):
    """{phase: warp clock cycles} of the last bit-packed traversal pass."""
    v = np.zeros(len(PHASES), np.int64)
    _chk(lib().cc_last_pass_phases(g, _p(v)), "cc_last_pass_phases")
    return dict(zip(PHASES, (int(x) for x in v)))


def cc_set_tuning(g, alpha=0):
    _chk(lib().cc_set_tuning(g, int(alpha)), "cc_set_tuning")


CC_PARAM_ALPHA, CC_PARAM_HYBRID_ONE_PASS, CC_PARAM_SSSP_DELTA, CC_PARAM_REACH_WORDS = 0, 1, 2, 3
CC_PARAM_ESTIMATE_GRAPH = 4


def cc_set_param(g, param, value):
    _chk(lib().cc_set_param(g, int(param), int(value)), "cc_set_param")


def cc_last_pass_trace(g, max_levels=64):
    """List of (level, ns, top_down, frontier, frontier_arcs, words) of the
    last traversal pass."""
    t = np.zeros(max_levels, np.int64)
    d = np.zeros(max_levels, np.int32)
    f = np.zeros(max_levels, np.int64)
    fa = np.zeros(max_levels, np.int64)
    wd = np.zeros(max_levels, np.int64)
    L = lib().cc_last_pass_trace(g, max_levels, _p(t), _p(d), _p(f), _p(fa), _p(wd))
    if L < 0:
        raise CCError(L, "cc_last_pass_trace")
    return [(l, int(t[l]), int(d[l]), int(f[l]), int(fa[l]), int(wd[l]))
            for l in range(1, L)]


def cc_last_call_timing(g):
    """(traversal launches, their kernel ms, alg bytes, all kernel launches)
    of the last traversal call on g."""
    n, a = ctypes.c_int32(), ctypes.c_int32()
    ms, b = ctypes.c_double(), ctypes.c_double()
    _chk(lib().cc_last_call_timing(g, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(b),
                                   ctypes.byref(a)), "cc_last_call_timing")
    return n.value, ms.value, b.value, a.value


def cc_last_call_graph(g):
    """True when the last cc_estimate on g replayed its captured CUDA graph."""
    r = ctypes.c_int32()
    _chk(lib().cc_last_call_graph(g, ctypes.byref(r)), "cc_last_call_graph")
    return bool(r.value)


def cc_sampling_pivots_noalloc(n, d_row_ptr, d_col, sample, d_sample_sum, d_pivot,
                               d_delta, d_S_sampled, stream=None):
    """Device pointers (ints) in, device pointers out; returns the status
    code (see include/cc.h: this call allocates nothing)."""
    sample = np.ascontiguousarray(sample, dtype=np.int32)
    return lib().cc_sampling_pivots_noalloc(int(n), d_row_ptr, d_col, _p(sample),
                                            sample.size, d_sample_sum, d_pivot, d_delta,
                                            d_S_sampled, stream)


def cc_selftest_barrier_timeout(timeout_ns):
    return lib().cc_selftest_barrier_timeout(ctypes.c_uint64(int(timeout_ns)))


# ---------------------------------------------------------------- batches

def cc_batch_create(graphs, samples, eps=None, autotune=True):
    """graphs: list of handles; samples: list of int32 arrays; eps: list of
    (num, den) or None."""
    ng = len(graphs)
    hs = (ctypes.c_void_p * ng)(*graphs)
    arrs = [np.ascontiguousarray(s, dtype=np.int32) for s in samples]
    ptrs = (ctypes.c_void_p * ng)(*[a.ctypes.data for a in arrs])
    ks = np.array([a.size for a in arrs], dtype=np.int32)
    num = den = None
    if eps is not None:
        num = np.array([e[0] for e in eps], dtype=np.uint32)
        den = np.array([e[1] for e in eps], dtype=np.uint32)
    b = ctypes.c_void_p()
    _chk(lib().cc_batch_create(ng, hs, ptrs, _p(ks), _p(num), _p(den), int(autotune),
                               ctypes.byref(b)), "cc_batch_create")
    return b.value


def cc_batch_run(b, stream=None):
    _chk(lib().cc_batch_run(b, stream), "cc_batch_run")


def cc_batch_result(b, i, n, k):
    """Host copies of graph i's results (same dict as cc_estimate)."""
    res = dict(s_hat=np.zeros((CC_NUM_EST, n)), closeness=np.zeros((CC_NUM_EST, n)),
               pivot=np.empty(n, np.int32), delta=np.empty(n, np.uint32),
               sum=np.empty(n, np.uint64), hyb=np.zeros((n, 6), np.uint64),
               S_samp=np.empty(k, np.uint64), delta_cc=np.empty((k, k), np.uint32))
    o = cc_out()
    for e in range(CC_NUM_EST):
        o.s_hat[e] = _p(res["s_hat"][e])
        o.closeness[e] = _p(res["closeness"][e])
    o.pivot, o.delta = _p(res["pivot"]), _p(res["delta"])
    o.sample_sum, o.hyb_int = _p(res["sum"]), _p(res["hyb"])
    o.S_sampled, o.delta_cc = _p(res["S_samp"]), _p(res["delta_cc"])
    _chk(lib().cc_batch_result(b, int(i), ctypes.byref(o), 0), "cc_batch_result")
    return res


def cc_batch_info(b):
    t, g, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    ms = ctypes.c_double()
    _chk(lib().cc_batch_info(b, ctypes.byref(t), ctypes.byref(g), ctypes.byref(ms),
                             ctypes.byref(c)), "cc_batch_info")
    return dict(teams=t.value, grid=g.value, last_ms=ms.value, graph_captured=bool(c.value))


def cc_batch_plan(b, i):
    """Graph i's plan: word width, alpha, team, class teams, class CTAs,
    CTAs per SM, tuning taken from the autotune cache."""
    v = [ctypes.c_int32() for _ in range(7)]
    _chk(lib().cc_batch_plan(b, int(i), *[ctypes.byref(x) for x in v]), "cc_batch_plan")
    return dict(zip(("words", "alpha", "team", "class_teams", "class_ctas", "ctas_per_sm",
                     "from_cache"), (x.value for x in v)))


def cc_batch_tune_cache(path):
    """Autotune cache file of cc_batch_create (None: off)."""
    _chk(lib().cc_batch_tune_cache(None if path is None else str(path).encode()),
         "cc_batch_tune_cache")


def cc_batch_free(b):
    _chk(lib().cc_batch_free(b), "cc_batch_free")


# ---------------------------------------------------------------- serving

def cc_server_create(graphs, slots=4, hbm_budget=0):
    hs = (ctypes.c_void_p * len(graphs))(*graphs)
    h = ctypes.c_void_p()
    _chk(lib().cc_server_create(len(graphs), hs, int(slots), ctypes.c_uint64(hbm_budget),
                                ctypes.byref(h)), "cc_server_create")
    return h.value


def cc_server_submit(s, graph, estimator, k, seed, eps=None):
    a, b = eps if eps is not None else (1, max(1, int(round(k ** 0.5))))
    rid = ctypes.c_int64()
    _chk(lib().cc_server_submit(s, int(graph), int(estimator), int(k),
                                ctypes.c_uint64(seed & (2**64 - 1)), a, b, ctypes.byref(rid)),
         "cc_server_submit")
    return rid.value


def cc_server_wait(s, rid, timeout_ms=60000):
    """Returns the status code (CC_OK, an error, or CC_ERR_TIMEOUT)."""
    return lib().cc_server_wait(s, int(rid), int(timeout_ms))


def cc_server_result(s, rid, n):
    out = dict(s_hat=np.empty(n), closeness=np.empty(n), pivot=np.empty(n, np.int32),
               delta=np.empty(n, np.uint32), sum=np.empty(n, np.uint64))
    lat = ctypes.c_double()
    _chk(lib().cc_server_result(s, int(rid), _p(out["s_hat"]), _p(out["closeness"]),
                                _p(out["pivot"]), _p(out["delta"]), _p(out["sum"]),
                                ctypes.byref(lat)), "cc_server_result")
    out["latency_ms"] = lat.value
    return out


def cc_server_stats(s):
    c, pk = ctypes.c_int64(), ctypes.c_int32()
    p50, p99, mean = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _chk(lib().cc_server_stats(s, ctypes.byref(c), ctypes.byref(p50), ctypes.byref(p99),
                               ctypes.byref(mean), ctypes.byref(pk)), "cc_server_stats")
    return dict(completed=c.value, p50_ms=p50.value, p99_ms=p99.value, mean_ms=mean.value,
                peak_running=pk.value)


def cc_server_cache_stats(s):
    h, m, n = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    b = ctypes.c_uint64()
    _chk(lib().cc_server_cache_stats(s, ctypes.byref(h), ctypes.byref(m), ctypes.byref(n),
                                     ctypes.byref(b)), "cc_server_cache_stats")
    return dict(hits=h.value, misses=m.value, states=n.value, resident_bytes=b.value)


def cc_server_free(s):
    _chk(lib().cc_server_free(s), "cc_server_free")
