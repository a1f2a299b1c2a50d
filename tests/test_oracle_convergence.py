"""Pins of the oracle's convergence decision (the paper asks that skill rise
with L over the r realizations but states no test; the reading here is a
Jonckheere-Terpstra trend test over the L groups, one-sided).

Pinned against: the statistic's extreme values, a sum of Mann-Whitney U
statistics (scipy), the exact null mean and variance by enumerating every
permutation of a small sample, invariance to the order of the L axis, NaN
handling, and the coupled logistic map (converges) against independent maps
(does not).
"""

from __future__ import annotations

import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1905_00565_gb300 import inputs as I


def jt_count(groups):
    """J by its definition: pairs (x in an earlier group, y in a later one),
    1 when y > x, 1/2 when equal."""
    J = 0.0
    for a in range(len(groups)):
        for b in range(a + 1, len(groups)):
            for x in groups[a]:
                for y in groups[b]:
                    J += 1.0 if y > x else (0.5 if y == x else 0.0)
    return J


def test_extremes_of_the_statistic():
    L = np.array([10, 20, 40])
    up = np.array([[0.1, 0.2], [0.3, 0.4], [0.5, 0.6]])
    c = oracle.convergence(up, L)
    assert c[2] == 12.0 and c[3] > 0 and c[5] == 1.0        # J = 2*2 * 3 pairs of groups
    assert c[0] == pytest.approx(0.15) and c[1] == pytest.approx(0.55) and c[4] == 6
    down = up[::-1].copy()
    c = oracle.convergence(down, L)
    assert c[2] == 0.0 and c[3] < 0 and c[5] == 0.0
    assert c[3] == pytest.approx(-oracle.convergence(up, L)[3])


def test_j_is_a_sum_of_mann_whitney_u():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(4)
    rho = rng.normal(size=(5, 30)).round(1)       # rounding makes cross-group ties
    L = np.array([5, 10, 20, 40, 80])
    want = 0.0
    for a in range(5):
        for b in range(a + 1, 5):
            want += stats.mannwhitneyu(rho[b], rho[a], method="asymptotic").statistic
    assert oracle.convergence(rho, L)[2] == want
    assert oracle.convergence(rho, L)[2] == jt_count(list(rho))


def test_null_mean_and_variance_by_enumeration():
    """Groups of sizes 2, 3, 2 over distinct values: every assignment of the 7
    values to the groups is equally likely with no trend.  The oracle's z is
    (J - E[J]) / sqrt(Var[J]) with E and Var of that exact distribution."""
    vals = [0.11, 0.52, 0.23, 0.74, 0.35, 0.96, 0.47]
    sizes = [2, 3, 2]
    js = []
    for perm in itertools.permutations(vals):
        g = [perm[0:2], perm[2:5], perm[5:7]]
        js.append(jt_count(g))
    js = np.array(js)
    mean, var = js.mean(), js.var()
    # a row with r = 3 and the middle-size trick: pad groups 1 and 3 with NaN
    row = np.array([[0.52, 0.11, np.nan], [0.74, 0.23, 0.35], [0.96, 0.47, np.nan]])
    c = oracle.convergence(row, np.array([1, 2, 3]))
    J = jt_count([[0.52, 0.11], [0.74, 0.23, 0.35], [0.96, 0.47]])
    assert c[2] == J and c[4] == sum(sizes)
    assert c[3] == pytest.approx((J - mean) / math.sqrt(var), rel=1e-12)


def test_order_of_the_l_axis_does_not_matter():
    rng = np.random.default_rng(7)
    rho = rng.normal(size=(3, 4, 6, 25))          # 12 rows of 6 L values
    L = np.array([100, 200, 400, 800, 1600, 3200])
    perm = np.array([3, 0, 5, 1, 4, 2])
    a = oracle.convergence(rho, L)
    b = oracle.convergence(rho[:, :, perm, :], L[perm])
    np.testing.assert_array_equal(a, b)


def test_nan_realizations_are_left_out():
    rho = np.array([[0.1, np.nan, 0.2], [0.4, 0.5, np.nan]])
    c = oracle.convergence(rho, np.array([10, 20]))
    assert c[4] == 4 and c[2] == 4.0 and c[0] == pytest.approx(0.15) and c[1] == pytest.approx(0.45)


def test_coupled_logistic_converges_and_independent_maps_do_not():
    n = 500
    s = I.logistic_pair(n)                        # y is driven by x (b_yx = 0.1)
    L = np.array([15, 40, 100, 250, 495], np.int64)
    rho = oracle.ccm(s, [[1, 0]], [2], [1], L, 12, seed=3)   # cross-map x from M_y
    c = oracle.convergence(rho, L)[0, 0, 0]
    assert c[5] == 1.0 and c[3] > 3.0 and c[1] > 0.5
    rng = np.random.default_rng(9)
    ind = np.stack([rng.random(n), rng.random(n)]).astype(np.float32)   # no coupling at all
    rho0 = oracle.ccm(ind, [[1, 0]], [2], [1], L, 12, seed=3)
    c0 = oracle.convergence(rho0, L)[0, 0, 0]
    assert c0[5] == 0.0 and abs(c0[1]) < 0.2
