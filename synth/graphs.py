"""Edge-list generators driven by a counter-based splitmix64 stream.

Random draws use splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) in counter form: the c-th value
(c = 0, 1, 2, ...) of stream `seed` is mix(seed + (c+1) * 0x9E3779B97F4A7C15),
where mix is the splitmix64 output function.  Every value therefore depends
only on (seed, c), so the graphs are identical on every machine.

All generators return (n, src, dst) with uint32 endpoint arrays of equal
length; weighted generators also return uint32 weights.  Duplicates and
self-loops are left in -- removing them is part of building the graph.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 23


def splitmix64_at(seed: int, counters) -> np.ndarray:
    """splitmix64 outputs number `counters` (uint64 array) of stream `seed`."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_at(seed: int, counters) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of splitmix64_at."""
    return (splitmix64_at(seed, counters) >> np.uint64(11)).astype(np.float64) * (
        1.0 / 9007199254740992.0
    )


def rmat_edges(scale: int, edge_factor: int, a=0.57, b=0.19, c=0.19, seed=1,
               relabel=True):
    """Graph500-style R-MAT edge list without noise.

    n = 2**scale nodes and edge_factor * n edges.  For edge e and bit level
    l (most significant first) the draw uniform_at(seed, e*scale + l) picks a
    quadrant: [0,a) -> (0,0), [a,a+b) -> (0,1), [a+b,a+b+c) -> (1,0), else
    (1,1), giving one bit of the source and one of the destination.  With
    `relabel`, node v is renamed to its rank under the keys
    splitmix64_at(seed + 1, v) (ties by v), which scatters the hubs.
    """
    n = 1 << scale
    m = edge_factor * n
    src = np.zeros(m, dtype=np.uint32)
    dst = np.zeros(m, dtype=np.uint32)
    # u = x * 2^-53 with x = (splitmix64 output) >> 11, so u >= t exactly
    # when x >= ceil(t * 2^53): the quadrant tests run on integers.
    t_ab, t_abc = a + b, a + b + c
    X_a, X_ab, X_abc = (np.uint64(math.ceil(t * 2.0 ** 53)) for t in (a, t_ab, t_abc))
    sd = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for lo in range(0, m, _CHUNK):
            hi = min(m, lo + _CHUNK)
            e = np.arange(lo, hi, dtype=np.uint64)
            s = np.zeros(hi - lo, dtype=np.uint32)
            d = np.zeros(hi - lo, dtype=np.uint32)
            # splitmix64 state seed + (counter + 1) * gamma for counter
            # e * scale + lev, advanced by gamma per level
            zc = sd + (e * np.uint64(scale) + np.uint64(1)) * _GAMMA
            z = np.empty_like(zc)
            t = np.empty_like(zc)
            for lev in range(scale):
                np.right_shift(zc, np.uint64(30), out=t)
                np.bitwise_xor(zc, t, out=z)
                z *= _M1
                np.right_shift(z, np.uint64(27), out=t)
                z ^= t
                z *= _M2
                np.right_shift(z, np.uint64(31), out=t)
                z ^= t
                z >>= np.uint64(11)
                shift = np.uint32(scale - 1 - lev)
                hi_s = z >= X_ab
                s |= hi_s.astype(np.uint32) << shift
                d |= (((z >= X_a) & ~hi_s) | (z >= X_abc)).astype(np.uint32) << shift
                zc += _GAMMA
            src[lo:hi] = s
            dst[lo:hi] = d
    if relabel:
        keys = splitmix64_at(seed + 1, np.arange(n, dtype=np.uint64))
        order = np.lexsort((np.arange(n), keys))
        new_id = np.empty(n, dtype=np.uint32)
        new_id[order] = np.arange(n, dtype=np.uint32)
        src = new_id[src]
        dst = new_id[dst]
    return n, src, dst


def grid_edges(width: int, height: int):
    """4-neighbour width x height grid; node (x, y) has id y*width + x."""
    n = width * height
    ids = np.arange(n, dtype=np.uint32).reshape(height, width)
    hs, hd = ids[:, :-1].ravel(), ids[:, 1:].ravel()
    vs, vd = ids[:-1, :].ravel(), ids[1:, :].ravel()
    return n, np.concatenate([hs, vs]), np.concatenate([hd, vd])


def watts_strogatz_edges(n: int, degree: int = 10, p: float = 0.05, seed=1):
    """Watts-Strogatz small world: ring lattice where node u links to
    u+1..u+degree/2 (mod n); each such edge keeps u and, with probability p
    (draw uniform_at(seed, 2t)), moves its far end to the node
    floor(uniform_at(seed, 2t+1) * n), t being the edge's index."""
    half = degree // 2
    u = np.repeat(np.arange(n, dtype=np.uint64), half)
    j = np.tile(np.arange(1, half + 1, dtype=np.uint64), n)
    v = (u + j) % np.uint64(n)
    t = np.arange(u.size, dtype=np.uint64)
    rew = uniform_at(seed, np.uint64(2) * t) < p
    tgt = np.minimum((uniform_at(seed, np.uint64(2) * t + np.uint64(1)) * n)
                     .astype(np.uint64), np.uint64(n - 1))
    v = np.where(rew, tgt, v)
    return n, u.astype(np.uint32), v.astype(np.uint32)


def rgg_edges(n: int, radius: float, seed=1):
    """Random geometric graph: n points uniform on the unit square (x from
    uniform_at(seed, 2i), y from uniform_at(seed, 2i+1)); an edge joins every
    pair closer than `radius`.  Returns (n, src, dst, length) with float64
    Euclidean lengths."""
    i = np.arange(n, dtype=np.uint64)
    x = uniform_at(seed, np.uint64(2) * i)
    y = uniform_at(seed, np.uint64(2) * i + np.uint64(1))
    g = max(1, int(np.floor(1.0 / radius)))
    cx = np.minimum((x * g).astype(np.int64), g - 1)
    cy = np.minimum((y * g).astype(np.int64), g - 1)
    cell = cy * g + cx
    order = np.argsort(cell, kind="stable")
    cell_sorted = cell[order]
    start = np.searchsorted(cell_sorted, np.arange(g * g + 1))
    count = np.diff(start)
    srcs, dsts, lens = [], [], []
    r2 = radius * radius
    pos = np.arange(n)  # position in sorted order
    pcx, pcy = cx[order], cy[order]
    for dx, dy in ((0, 0), (1, 0), (-1, 1), (0, 1), (1, 1)):
        ncx, ncy = pcx + dx, pcy + dy
        ok = (ncx >= 0) & (ncx < g) & (ncy < g)
        a_pos = pos[ok]
        b_cell = (ncy * g + ncx)[ok]
        reps = count[b_cell]
        tot = int(reps.sum())
        if tot == 0:
            continue
        a_rep = np.repeat(a_pos, reps)
        first = np.repeat(start[b_cell], reps)
        seg_start = np.repeat(np.cumsum(reps) - reps, reps)
        b_rep = first + (np.arange(tot) - seg_start)
        if dx == 0 and dy == 0:
            keep = b_rep > a_rep
            a_rep, b_rep = a_rep[keep], b_rep[keep]
        ia, ib = order[a_rep], order[b_rep]
        d2 = (x[ia] - x[ib]) ** 2 + (y[ia] - y[ib]) ** 2
        close = d2 < r2
        srcs.append(ia[close].astype(np.uint32))
        dsts.append(ib[close].astype(np.uint32))
        lens.append(np.sqrt(d2[close]))
    return (n, np.concatenate(srcs), np.concatenate(dsts),
            np.concatenate(lens))


def edge_lengths_to_weights(lengths, scale: float = 1000.0) -> np.ndarray:
    """uint32 arc lengths round(scale * length) + 1 (always >= 1)."""
    return (np.rint(np.asarray(lengths) * scale) + 1).astype(np.uint32)


def random_weights(m: int, lo: int, hi: int, seed=1) -> np.ndarray:
    """m uint32 weights uniform on [lo, hi] from uniform_at(seed, e)."""
    u = uniform_at(seed, np.arange(m, dtype=np.uint64))
    return (lo + np.minimum((u * (hi - lo + 1)).astype(np.int64), hi - lo)).astype(
        np.uint32)


def pareto_node_weights(n: int, alpha: float = 1.2, scale: int = 10, cap: int = 10**6,
                        seed=1) -> np.ndarray:
    """n uint32 node weights min(cap, floor(scale * x) + 1), x Pareto (Lomax)
    of shape alpha from uniform_at(seed, v): a few heavy nodes among many
    light ones."""
    u = uniform_at(seed, np.arange(n, dtype=np.uint64))
    x = (1.0 - u) ** (-1.0 / alpha) - 1.0
    return np.minimum(np.floor(scale * x) + 1, cap).astype(np.uint32)


def path_edges(n: int):
    """Path 0 - 1 - ... - (n-1)."""
    a = np.arange(n - 1, dtype=np.uint32)
    return n, a, a + np.uint32(1)


def star_edges(n: int):
    """Star K_{1,n-1} with centre 0."""
    return n, np.zeros(n - 1, dtype=np.uint32), np.arange(1, n, dtype=np.uint32)


def cycle_edges(n: int):
    """Cycle 0 - 1 - ... - (n-1) - 0."""
    a = np.arange(n, dtype=np.uint32)
    return n, a, (a + np.uint32(1)) % np.uint32(n)


def complete_edges(n: int):
    """Complete graph K_n (each pair once)."""
    iu, ju = np.triu_indices(n, 1)
    return n, iu.astype(np.uint32), ju.astype(np.uint32)


def road_like_edges(n: int, mean_degree: float = 2.6, gen_degree: float = 5.0, seed=1):
    """Road-like graph: a random geometric graph on the unit square generated
    at mean degree `gen_degree` (above the 2-D percolation threshold, so one
    component spans the square), thinned to about `mean_degree`: a random
    spanning forest (minimum spanning forest under the random keys
    uniform_at(seed + 2, e)) is always kept and every other edge is kept with
    the probability that brings the mean degree to `mean_degree` (draw
    uniform_at(seed + 3, e)).  Returns (n, src, dst, length)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import minimum_spanning_tree

    radius = float(np.sqrt(gen_degree / (np.pi * n)))
    n, src, dst, length = rgg_edges(n, radius, seed=seed)
    m = src.size
    key = uniform_at(seed + 2, np.arange(m, dtype=np.uint64)) + 1e-9
    g = coo_matrix((key, (src.astype(np.int64), dst.astype(np.int64))), shape=(n, n))
    forest = minimum_spanning_tree(g.tocsr()).tocoo()
    fpair = np.minimum(forest.row, forest.col).astype(np.int64) * n + \
        np.maximum(forest.row, forest.col).astype(np.int64)
    upair = np.minimum(src, dst).astype(np.int64) * n + np.maximum(src, dst).astype(np.int64)
    in_forest = np.isin(upair, fpair)
    extra_needed = max(0.0, mean_degree * n / 2.0 - in_forest.sum())
    q = min(1.0, extra_needed / max(1, (~in_forest).sum()))
    keep = in_forest | (uniform_at(seed + 3, np.arange(m, dtype=np.uint64)) < q)
    return n, src[keep], dst[keep], length[keep]
