"""Helpers of the full-size parity tests: the oracle's searches run in
threads (its C routines release the interpreter lock), and the nodes to
check are picked across degree classes so that hubs and the nodes of every
traversal path are among them."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from oracle import oracle as orc

THREADS = max(1, min(32, os.cpu_count() or 1))


def pmap(fn, items):
    items = list(items)
    with ThreadPoolExecutor(THREADS) as ex:
        return list(ex.map(fn, items))


def dist_table(og, sources, roundtrip=False):
    """orc.dist_table with the sources split across threads."""
    src = np.ascontiguousarray(sources, dtype=np.int32)
    chunks = [c for c in np.array_split(src, min(THREADS, src.size)) if c.size]
    return np.concatenate(pmap(lambda c: orc.dist_table(og, c, roundtrip), chunks), axis=0)


def picks(degree, sample, seed, hubs=20, per_class=45, bounds=(4, 32, 256), extra=()):
    """Sorted distinct nodes: the `hubs` highest degrees, `per_class`
    random nodes from each degree class (<= 4, <= 32, <= 256, larger: the
    tiny, light, medium and heavy nodes of the traversal), the first and
    last sampled nodes and `extra`."""
    deg = np.asarray(degree)
    rng = np.random.default_rng(seed)
    out = set(np.argsort(-deg, kind="stable")[:hubs].tolist())
    lo = -1
    for hi in list(bounds) + [int(deg.max())]:
        cls = np.flatnonzero((deg > lo) & (deg <= hi))
        if cls.size:
            out.update(rng.choice(cls, min(per_class, cls.size), replace=False).tolist())
        lo = hi
    out.update([int(sample[0]), int(sample[-1])])
    out.update(int(x) for x in extra)
    return sorted(out)


def rel_close(got, want, tol=1e-12):
    return abs(got - want) <= tol * abs(want)
