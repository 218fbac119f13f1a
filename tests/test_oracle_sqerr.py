"""Pins of the oracle's error estimate SqErrEst and the adaptive hybrid.

SqErrEst(v) (Algorithm 1's last loop; section 4, eqs. (5) and (6)) is
  |L| / |L n C| * var(L n C) + |H| * SQ(H),
var the sample variance of d(c_i, v) over c_i in L(v) n C and SQ the mean
of (d(c_i, v) - d(c(v), c_i))^2 over c_i in HC(v); when HC(v) is empty the
farthest sampled node from c(v) stands in.  The adaptive hybrid (section 6)
keeps, per node, the eps with the smallest SqErrEst.

Every expected value below is a closed form derived by hand on small paths,
a star and a cycle, not a re-evaluation of the oracle's formulas.
"""
import numpy as np
import pytest

import synth
from oracle import oracle as O


def _path_table(n, C):
    g = O.csr_from_edges(*synth.path_edges(n))
    return O.dist_table(g, np.asarray(C, np.int32))


@pytest.mark.parametrize("n", [20, 31])
def test_pivot_term_only_path(n):
    # Path 0..n-1, C = {0, n-1}, eps = 1/2.  For 1 <= v < (n-1)/2 the pivot
    # is node 0 (Delta = v), the threshold 2v puts c = n-1 (at n-1 from the
    # pivot) in HC and leaves L n C = {0}: one sample, variance 0.  H = the
    # nodes at distance > 2v from 0 other than n-1: |H| = n-2-2v.  SQ =
    # (d(n-1, v) - d(0, n-1))^2 = ((n-1-v) - (n-1))^2 = v^2.
    C = [0, n - 1]
    _, se = O.sqerr_from_table(_path_table(n, C), C, (1, 2))
    for v in range(1, (n - 1) // 2):
        if n - 2 - 2 * v < 0:
            continue
        assert se[v] == v * v * (n - 2 - 2 * v), v


@pytest.mark.parametrize("n", [20, 30])
def test_both_terms_path(n):
    # Path, C = {0, 1, n-1}, v = 3, eps = 1/2: pivot node 1 (Delta 2),
    # threshold 4.  L n C = {0, 1} with distances {3, 2}: sum 5, squares
    # 13, so var * |L n C|^2 = 13*2 - 25 = 1.  HC = {n-1} (at n-2 > 4 from
    # the pivot); H = nodes 6..n-2 (|H| = n-7); |L| = (n-1) - (n-7) - 1 = 5.
    # Sampling term 1 * 5 / 2^3 = 5/8.  Pivot term: (d(n-1, 3) -
    # d(1, n-1))^2 = ((n-4) - (n-2))^2 = 4, times |H|.
    C = [0, 1, n - 1]
    s_hat, se = O.sqerr_from_table(_path_table(n, C), C, (1, 2))
    assert se[3] == pytest.approx(5 / 8 + 4 * (n - 7), rel=1e-15)
    # Estimate, eq. (4): Hsum = sum of d(1, w), w = 6..n-2, = sum 5..n-3;
    # HCsum = d(n-1, 3) = n-4; sampling part 5 * |L| / |L n C| = 25/2.
    hsum = sum(range(5, n - 2))
    assert s_hat[3] == pytest.approx(hsum + (n - 4) + 12.5, rel=1e-15)


@pytest.mark.parametrize("n", [16, 25])
def test_empty_hc_falls_back_to_farthest_sample(n):
    # Path, C = {0, 1}, v = 5, eps = 1/2: pivot node 1 (Delta 4), threshold
    # 8; no sampled node lies beyond it (HC empty) but H = nodes 10..n-1
    # does (|H| = n-10).  The farthest sampled node from the pivot other
    # than itself is node 0 (at 1): SQ = (d(0, 5) - 1)^2 = 16.  L n C =
    # {0, 1}, distances {5, 4}: var * 4 = 41*2 - 81 = 1; |L| = 9.
    C = [0, 1]
    _, se = O.sqerr_from_table(_path_table(n, C), C, (1, 2))
    assert se[5] == pytest.approx(9 / 8 + 16 * (n - 10), rel=1e-15)


@pytest.mark.parametrize("n,k", [(10, 4), (33, 7)])
def test_sampling_term_star_closed_form(n, k):
    # Star, centre 0, leaves 1..n-1; C = {0, 1, ..., k-1}; v = a leaf not in
    # C.  With eps = 1/1000 nothing is beyond the threshold 1000 * Delta, so
    # H and HC are empty and L n C = C with distances {1, 2 x (k-1)}:
    # var * k^2 = (4k-3) k - (2k-1)^2 = k - 1; |L| = n - 1.
    C = list(range(k))
    g = O.csr_from_edges(*synth.star_edges(n))
    T = O.dist_table(g, np.asarray(C, np.int32))
    _, se = O.sqerr_from_table(T, C, (1, 1000))
    for v in range(k, n):
        assert se[v] == pytest.approx((k - 1) * (n - 1) / k ** 3, rel=1e-15)


def test_full_sample_has_no_error():
    # C = V: every node is sampled, every S is exact (section 2) and every
    # error estimate is 0; the adaptive choice is "none".
    n = 12
    g = O.csr_from_edges(*synth.cycle_edges(n))
    C = np.arange(n, dtype=np.int32)
    T = O.dist_table(g, C)
    s_hat, se = O.sqerr_from_table(T, C, (1, 3))
    s2, se2, ch = O.adaptive_from_table(T, C)
    exact = np.array([sum(min(abs(u - v), n - abs(u - v)) for u in range(n))
                      for v in range(n)], np.float64)
    assert np.array_equal(s_hat, exact) and np.array_equal(s2, exact)
    assert not se.any() and not se2.any()
    assert (ch == -1).all()


def test_adaptive_picks_smallest_error_path():
    # Path n = 20, C = {0, 1, 19}, v = 3 (pivot node 1, Delta 2), by hand
    # for each eps of the list (threshold t = 2/eps; x beyond iff x > t):
    #   0.99: HC = {19}, |H| = 15 (w = 4..18), |L| = 3: 3/8 + 4*15 = 60.375
    #   0.5 : HC = {19}, |H| = 13, |L| = 5:           5/8 + 4*13 = 52.625
    #   0.2 : HC = {19}, |H| = 7 (w = 12..18), |L| = 11: 11/8 + 28 = 29.375
    #   <= 0.1: HC empty, |H| = 0, L n C = C with distances {3, 2, 16}:
    #         var * 9 = 269*3 - 441 = 366; |L| = 19: 366*19/27 = 257.56
    # The smallest is eps = 0.2 (position 4); its estimate is Hsum (d(1, w),
    # w = 12..18: 11 + ... + 17 = 98) + HCsum (d(19, 3) = 16) + 5 * 11 / 2.
    C = [0, 1, 19]
    s_hat, se, ch = O.adaptive_from_table(_path_table(20, C), C)
    assert ch[3] == 4
    assert se[3] == pytest.approx(29.375, rel=1e-15)
    assert s_hat[3] == pytest.approx(98 + 16 + 27.5, rel=1e-15)


def test_sqerr_estimate_matches_hybrid_of_estimate():
    # The same eq. (4) estimate comes out of both oracle entry points.
    g = O.csr_from_edges(*synth.rmat_edges(9, 8, seed=3))
    C = O.choose_sample(g.n, 24, 5)
    T = O.dist_table(g, C)
    s_hat, _ = O.sqerr_from_table(T, C, (1, 5))
    ref = O.estimate_from_table(T, C, (1, 5))["s_hat"][3]
    assert np.array_equal(s_hat, ref)


def test_fallback_uses_the_farthest_sample():
    # Path 0..19 plus a pendant node 20 on node 10 (n = 21); C = {11, 12, 5};
    # v = 20, eps = 1/4.  d(c, 20) = 2, 3, 6, so the pivot is node 11
    # (Delta 2) and the threshold 8.  Sampled nodes lie 1 and 6 from the
    # pivot: HC is empty; H = {0, 1, 2} (11 - w > 8).  The farthest sampled
    # node from the pivot is node 5: SQ = (d(5, 20) - d(11, 5))^2 =
    # (6 - 6)^2 = 0 -- the nearer node 12 would give (3 - 1)^2 = 4.
    # Sampling term: distances {2, 3, 6}: var * 9 = 49*3 - 121 = 26, and
    # |L| = 20 - 3 - 0 = 17: 26 * 17 / 27.
    n0, s, d = synth.path_edges(20)
    s = np.append(s, np.uint32(10))
    d = np.append(d, np.uint32(20))
    g = O.csr_from_edges(21, s, d)
    C = [11, 12, 5]
    T = O.dist_table(g, np.asarray(C, np.int32))
    _, se = O.sqerr_from_table(T, C, (1, 4))
    assert se[20] == pytest.approx(26 * 17 / 27, rel=1e-15)
