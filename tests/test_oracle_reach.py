"""Pins of the oracle's outbound / inbound estimates for general directed
graphs (section 6.2, Algorithm 4): the average distance to a bottom-k sample
of each node's reachability set and the bottom-k estimate of its size.

The pins: closed forms on a directed path and a cycle; over every order of
a small graph the average distance is exactly unbiased and the size estimate
has the expectation 1 + (n-2) r / (n-1) derived by hand (r = |R(v)| >= k;
below k the count is exact); inbound is outbound on the reversed graph; and
the paper's own procedure -- pruned searches in rank order on the reversed
graph, with its mark rule for T -- computed independently gives the same
counts, sums and positions.
"""
from collections import deque
from fractions import Fraction
from itertools import permutations

import numpy as np
import pytest

import synth
from oracle import oracle as O


def digraph(n, arcs):
    s = np.array([a for a, _ in arcs], np.uint32)
    d = np.array([b for _, b in arcs], np.uint32)
    return O.csr_from_edges(n, s, d, directed=True, keep_component=False)


def small_dag():
    # 7 nodes: reach sets of different sizes, two paths of unequal length
    return digraph(7, [(0, 1), (1, 2), (2, 3), (0, 4), (4, 3), (3, 5), (6, 5), (5, 6),
                       (1, 4)])


@pytest.mark.parametrize("k", [3, 8, 40])
def test_directed_path_closed_form(k):
    n = 12
    g = digraph(n, [(i, i + 1) for i in range(n - 1)])
    r = O.reach_from_table(O.all_pairs(g), O.sample_order(n, 4), k)
    for v in range(n):
        reach = n - 1 - v
        if reach <= k:  # every reachable node sampled: exact sums
            assert r["count"][v] == reach
            assert int(r["distsum"][v]) == reach * (reach + 1) // 2
            if reach < k:  # fewer than k: the count is the size
                assert r["R_hat"][v] == reach
        else:
            assert r["count"][v] == k


def test_cycle_with_k_all_others_is_exact():
    # k = n - 1 on a directed cycle: every node reaches all n-1 others at
    # distances 1..n-1 (mean n/2), and the k-th sample is the last other
    # node in the order (T = n - 1), so R_hat = 1 + (n-2)(n-2)/(n-2) = n-1.
    n = 9
    g = digraph(n, [(i, (i + 1) % n) for i in range(n)])
    r = O.reach_from_table(O.all_pairs(g), O.sample_order(n, 1), n - 1)
    assert (r["T"] == n - 1).all()
    assert np.array_equal(r["R_hat"], np.full(n, n - 1.0))
    assert np.array_equal(r["avg"], np.full(n, n / 2))


@pytest.mark.parametrize("k", [2, 3])
def test_expectation_over_every_order(k):
    # Averaged over all 7! orders: avg is the exact mean distance over R(v)
    # (the sample is a uniform k-subset of R(v)); R_hat has expectation
    # 1 + (n-2) r/(n-1), from E[(k-1)/(T-1)] = r/(n-1) for the position T
    # of the k-th of r marked nodes among the n-1 others.
    g = small_dag()
    n = g.n
    D = O.all_pairs(g)
    acc_avg = [Fraction(0)] * n
    acc_R = [Fraction(0)] * n
    perms = list(permutations(range(n)))
    for order in perms:
        r = O.reach_from_table(D, order, k)
        for v in range(n):
            if r["count"][v] == k:
                acc_avg[v] += Fraction(int(r["distsum"][v]), k)
                acc_R[v] += 1 + Fraction((k - 1) * (n - 2), int(r["T"][v]) - 1)
            else:
                acc_R[v] += int(r["count"][v])
    for v in range(n):
        reach = [u for u in range(n) if u != v and D[v, u] != O.INF]
        rr = len(reach)
        if rr >= k:
            assert acc_avg[v] / len(perms) == Fraction(sum(int(D[v, u]) for u in reach), rr)
            assert acc_R[v] / len(perms) == 1 + Fraction((n - 2) * rr, n - 1)
        else:
            assert acc_R[v] / len(perms) == rr


def test_inbound_is_outbound_of_the_reversed_graph():
    n, s, d = synth.rmat_edges(7, 4, seed=5)
    g = O.csr_from_edges(n, s, d, directed=True, keep_component=False)
    gr = O.csr_from_edges(n, d, s, directed=True, keep_component=False)
    order = O.sample_order(g.n, 3)
    a = O.reach_from_table(O.all_pairs(g), order, 5, inbound=True)
    b = O.reach_from_table(O.all_pairs(gr), order, 5)
    for key in ("count", "distsum", "T"):
        assert np.array_equal(a[key], b[key])


def _pruned_searches(g, order, k):
    """Algorithm 4's procedure: BFS from each node in rank order on the
    reversed graph, pruned at saturated nodes, with the mark rule for T.
    The pruning counts the searches that reached a node including its own
    and prunes at k + 1: then a node x it stops at holds k + 1 nodes of
    smaller rank than u among x and its reachability set, and every node
    reaching x already has k of them other than itself."""
    n = g.n
    rp, col = g.rrow_ptr, g.rcol
    count = [0] * n
    seen = [0] * n  # searches that reached the node, its own included
    dsum = [0] * n
    T = [0] * n
    mark = [False] * n
    for t, u in enumerate(order, start=1):
        mark[u] = True
        dist = {u: 0}
        q = deque([u])
        while q:
            v = q.popleft()
            if seen[v] == k + 1:
                continue  # pruned: not scanned further
            seen[v] += 1
            if v != u and count[v] < k:
                dsum[v] += dist[v]
                count[v] += 1
                if count[v] == k:
                    T[v] = t - 1 if mark[v] else t
            for e in range(rp[v], rp[v + 1]):
                w = int(col[e])
                if w not in dist:
                    dist[w] = dist[v] + 1
                    q.append(w)
    return count, dsum, T


def test_pruning_on_other_nodes_alone_can_lose_a_sample():
    # The procedure as printed prunes at a node x once k nodes other than x
    # reached it.  On this graph with k = 1: 0 <-> 1, 2 -> 1, order 1, 0,
    # 2 ...: the search from 1 reaches 0 (0's sample {1}) and 2; the search
    # from 0 is pruned at 0 itself (full), so 1 -- whose reachability set
    # is {0} -- never receives 0.  The definition gives 1 the sample {0}.
    g = digraph(3, [(0, 1), (1, 0), (2, 1)])
    r = O.reach_from_table(O.all_pairs(g), [1, 0, 2], 1)
    assert r["count"].tolist() == [1, 1, 1]
    count, _, _ = _pruned_searches(g, [1, 0, 2], 1)
    assert count == [1, 1, 1]


@pytest.mark.parametrize("k", [1, 2, 4, 7])
def test_definition_matches_the_pruned_search(k):
    n, s, d = synth.rmat_edges(7, 3, seed=9)
    g = O.csr_from_edges(n, s, d, directed=True, keep_component=False)
    order = O.sample_order(g.n, 2)
    r = O.reach_from_table(O.all_pairs(g), order, k)
    count, dsum, T = _pruned_searches(g, [int(x) for x in order], k)
    assert r["count"].tolist() == count
    assert [int(x) for x in r["distsum"]] == dsum
    assert r["T"].tolist() == T


def test_weighted_directed_path_closed_form():
    # Arc lengths: path i -> i+1 of length len[i]; every node reaches the
    # higher ids at the prefix-sum distances.  k at least the reach: the
    # sums are exact.
    n = 10
    lens = [3, 1, 4, 1, 5, 9, 2, 6, 5]
    s = np.arange(n - 1, dtype=np.uint32)
    g = O.csr_from_edges(n, s, s + 1, w=np.array(lens, np.uint32), directed=True,
                         keep_component=False)
    r = O.reach_from_table(O.all_pairs(g), O.sample_order(n, 5), n)
    pre = np.concatenate([[0], np.cumsum(lens)])
    for v in range(n):
        want = sum(int(pre[u] - pre[v]) for u in range(v + 1, n))
        assert r["count"][v] == n - 1 - v
        assert int(r["distsum"][v]) == want


def test_weighted_sample_distances_are_shortest_paths():
    # With arc lengths the sample is still the k smallest ranks of R(v)
    # (lengths do not change reachability) and each sampled distance is the
    # shortest-path length; checked against scipy's Dijkstra.
    import scipy.sparse as sp
    from scipy.sparse.csgraph import shortest_path
    n, s, d = synth.rmat_edges(7, 4, seed=11)
    w = synth.random_weights(s.size, 1, 9, seed=12)
    g = O.csr_from_edges(n, s, d, w=w, directed=True, keep_component=False)
    A = sp.csr_matrix((g.w.astype(float), g.col, g.row_ptr), shape=(g.n, g.n))
    D = shortest_path(A, directed=True)
    order = [int(x) for x in O.sample_order(g.n, 4)]
    k = 5
    r = O.reach_from_table(O.all_pairs(g), order, k)
    for v in range(g.n):
        reach = [u for u in order if u != v and np.isfinite(D[v, u])][:k]
        assert r["count"][v] == len(reach)
        assert int(r["distsum"][v]) == int(sum(D[v, u] for u in reach))


def _group_schedule(g, order, k, G, inbound=False):
    """The device's schedule, modelled on the CPU: sources in rank order in
    groups of G searched together (unit lengths: breadth-first by levels;
    arc lengths: label-correcting rounds), nodes saturated at the start of
    a group -- k + 1 sources other than the node reached it, or k and its
    own search has run -- neither entered nor expanded, the first arrival
    (shortest distance) of each source recorded, then every touched node
    takes its lowest-rank sources other than itself until it holds k."""
    n = g.n
    if inbound:
        rp, col, w = g.row_ptr, g.col, g.w
    else:
        rp, col, w = g.rrow_ptr, g.rcol, g.rw
    rank = {int(u): p for p, u in enumerate(order)}
    cnt, extra, dsum, T = [0] * n, [False] * n, [0] * n, [0] * n

    def saturated(x, base):
        return cnt[x] >= k and (extra[x] or rank[x] < base)

    for base in range(0, n, G):
        srcs = [int(u) for u in order[base:base + G]]
        dist = {}                      # (node, i) -> distance
        front = {}
        for i, s in enumerate(srcs):
            if not saturated(s, base):
                dist[(s, i)] = 0
                front.setdefault(s, set()).add(i)
        while front:
            nxt = {}
            for u, bits in front.items():
                for e in range(rp[u], rp[u + 1]):
                    x = int(col[e])
                    if saturated(x, base):
                        continue
                    ln = 1 if w is None else int(w[e])
                    for i in bits:
                        cand = dist[(u, i)] + ln
                        if cand < dist.get((x, i), 1 << 62):
                            dist[(x, i)] = cand
                            nxt.setdefault(x, set()).add(i)
            front = nxt
        touched = {}
        for (x, i), d in dist.items():
            touched.setdefault(x, {})[i] = d
        for x, got in touched.items():
            for i in sorted(got):
                if srcs[i] == x:
                    continue
                if cnt[x] < k:
                    dsum[x] += got[i]
                    cnt[x] += 1
                    if cnt[x] == k:
                        t = base + i + 1
                        T[x] = t - 1 if rank[x] < base + i else t
                else:
                    extra[x] = True
                    break
    return cnt, dsum, T


@pytest.mark.parametrize("G", [1, 3, 16, 64])
@pytest.mark.parametrize("k", [1, 2, 5])
@pytest.mark.parametrize("lengths", [False, True])
def test_group_schedule_equals_definition(G, k, lengths):
    # Searching G rank-ordered sources at once, with the pruning rule
    # applied only at group boundaries and every touched node keeping its
    # lowest ranks, gives the definition's samples, distances and T.
    n, s, d = synth.rmat_edges(7, 3, seed=21)
    w = synth.random_weights(s.size, 1, 6, seed=22) if lengths else None
    g = O.csr_from_edges(n, s, d, w=w, directed=True, keep_component=False)
    order = [int(x) for x in O.sample_order(g.n, 6)]
    D = O.all_pairs(g)
    for inbound in (False, True):
        r = O.reach_from_table(D, order, k, inbound=inbound)
        cnt, dsum, T = _group_schedule(g, order, k, G, inbound=inbound)
        assert r["count"].tolist() == cnt
        assert [int(x) for x in r["distsum"]] == dsum
        assert r["T"].tolist() == T


@pytest.mark.parametrize("lengths", [False, True])
def test_single_node_reach_equals_table(lengths):
    # One search per node (for graphs too large for an n x n table) gives
    # the table function's count, sum, T and estimates.
    n, s, d = synth.rmat_edges(8, 4, seed=31)
    w = synth.random_weights(s.size, 1, 9, seed=32) if lengths else None
    g = O.csr_from_edges(n, s, d, w=w, directed=True, keep_component=False)
    order = O.sample_order(g.n, 9)
    D = O.all_pairs(g)
    for inbound in (False, True):
        for k in (1, 3, 20):
            ref = O.reach_from_table(D, order, k, inbound=inbound)
            for v in range(0, g.n, 3):
                r = O.reach_node(g, order, v, k, inbound=inbound)
                assert (r["count"], r["distsum"], r["T"]) == (
                    ref["count"][v], int(ref["distsum"][v]), ref["T"][v])
                assert r["avg"] == ref["avg"][v] and r["R_hat"] == ref["R_hat"][v]
