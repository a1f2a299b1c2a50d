"""Pins of the oracle's two optional CCM variants (not in the paper; both off
by default): the exclusion (Theiler) window W and the simplex weight floor f.

Pinned against brute force written out here, closed forms on series whose
neighbours are known by construction, and the argument checks.
"""

from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_1905_00565_gb300 import inputs as I
from tests.test_oracle_pins import _sqdist32, _sqdist64, _tiny_series


def brute_neighbours_window(s, E, tau, lib, W):
    """E+1 nearest library points with |l - m| > W, by (FP32 d^2, index)."""
    n_m = len(s) - (E - 1) * tau
    out = []
    for m in range(n_m):
        cand = sorted((_sqdist32(s, E, tau, m, int(l)), int(l)) for l in lib
                      if abs(int(l) - m) > W)
        out.append([l for _, l in cand[:E + 1]])
    return np.array(out, dtype=np.int32)


@pytest.mark.parametrize("kind", ["uniform", "integers", "logistic"])
@pytest.mark.parametrize("W", [0, 1, 4])
def test_theiler_window_matches_brute_force(kind, W):
    rng = np.random.default_rng(31 + W)
    s = _tiny_series(kind, 60, rng)
    for E, tau in [(1, 1), (2, 3), (3, 2)]:
        n_m = len(s) - (E - 1) * tau
        L = int(rng.integers(E + 2 + 2 * W, n_m + 1))
        lib = np.sort(rng.choice(n_m, size=L, replace=False)).astype(np.int32)
        got = oracle.neighbours(s, E, tau, lib, theiler=W)
        assert np.array_equal(got, brute_neighbours_window(s, E, tau, lib, W))


def test_theiler_zero_is_the_papers_rule():
    rng = np.random.default_rng(2)
    s = _tiny_series("logistic", 80, rng)
    lib = np.sort(rng.choice(78, size=40, replace=False)).astype(np.int32)
    assert np.array_equal(oracle.neighbours(s, 3, 1, lib), oracle.neighbours(s, 3, 1, lib, theiler=0))


def test_theiler_window_on_a_ramp_closed_form():
    """E = 1 on s[t] = t (exact in FP32), full library: the candidates nearest
    to m are m-W-1 and m+W+1 (equal distance, lower index first), then
    m-W-2, m+W+2, ...; near the ends the list continues on the open side."""
    n, W, E = 40, 3, 1
    s = np.arange(n, dtype=np.float32)
    lib = np.arange(n, dtype=np.int32)
    got = oracle.neighbours(s, E, 1, lib, theiler=W)
    for m in range(n):
        order = sorted((abs(l - m), l) for l in range(n) if abs(l - m) > W)
        assert got[m].tolist() == [l for _, l in order[:E + 1]]
    assert got[20].tolist() == [16, 24]
    assert got[0].tolist() == [4, 5]


def test_weight_floor_closed_form():
    """E = 2, tau = 1: query point m = 0 at (0, 0) and neighbours m = 3, 6, 9
    at (0, 1), (0, -2), (0, 30), distances 1, 2, 30 by construction:
    u = (e^-1, e^-2, e^-30); with a floor f, u_i = max(u_i, f)."""
    s = np.array([0, 0, 99, 1, 0, 77, -2, 0, 55, 30, 0], np.float32)
    pts = {m: (float(s[m + 1]), float(s[m])) for m in range(len(s) - 1)}
    row = [3, 6, 9]
    assert [pts[0]] + [pts[m] for m in row] == [(0.0, 0.0), (0.0, 1.0), (0.0, -2.0), (0.0, 30.0)]
    nbr = np.tile(np.array(row, np.int32), (len(s) - 1, 1))   # row 0 is the one checked
    t = np.arange(len(s), dtype=np.float32) * 3.0 + 1.0      # target; Xhat uses t[m + 1]
    for f in (0.0, 1e-6, 0.05):
        u = [max(math.exp(-1.0), f), max(math.exp(-2.0), f), max(math.exp(-30.0), f)]
        want = (u[0] * 13.0 + u[1] * 22.0 + u[2] * 31.0) / sum(u)
        got = oracle.predict(s, t, 2, 1, nbr, weight_floor=f)[0]
        assert got == pytest.approx(want, rel=1e-15, abs=0)
    # the floor matters exactly when it exceeds a weight: here only e^-30
    assert oracle.predict(s, t, 2, 1, nbr, weight_floor=1e-6)[0] != \
        oracle.predict(s, t, 2, 1, nbr)[0]


def test_weight_floor_with_d1_zero():
    """d_1 = 0: u = (1 for d_i = 0, else 0) before the floor, (1, f) after
    (E = 1: neighbours m = 1 and 2 of query 0, at distances 0 and 3)."""
    s = np.array([0.0, 0.0, 3.0, 4.0, 9.0], np.float32)
    t = np.array([1.0, 2.0, 4.0, 8.0, 16.0], np.float32)
    E = 1
    nbr = np.array([[1, 2]] * 5, np.int32)
    for f in (0.0, 0.25):
        u = [1.0, f]
        want = (u[0] * 2.0 + u[1] * 4.0) / sum(u)
        assert oracle.predict(s, t, E, 1, nbr, weight_floor=f)[0] == pytest.approx(want, rel=1e-15)


def test_weight_floor_predictions_match_brute_force():
    rng = np.random.default_rng(12)
    s = I.logistic_pair(90)
    E, tau, f = 3, 2, 1e-3
    n_m = 90 - (E - 1) * tau
    lib = np.sort(rng.choice(n_m, size=30, replace=False)).astype(np.int32)
    nbr = oracle.neighbours(s[0], E, tau, lib)
    got = oracle.predict(s[0], s[1], E, tau, nbr, weight_floor=f)
    for m, row in enumerate(nbr):
        d = [math.sqrt(_sqdist64(s[0], E, tau, m, int(l))) for l in row]
        u = [max(math.exp(-x / d[0]), f) if d[0] > 0 else max(1.0 if x == 0 else 0.0, f) for x in d]
        want = sum(ui * float(s[1][int(l) + (E - 1) * tau]) for ui, l in zip(u, row)) / sum(u)
        assert got[m] == pytest.approx(want, rel=1e-13)


def test_options_change_rho_and_zero_options_do_not():
    s = I.logistic_pair(300)
    base = oracle.ccm_unit(s, 1, 0, 3, 1, 120, 0, 7)
    assert oracle.ccm_unit(s, 1, 0, 3, 1, 120, 0, 7, theiler=0, weight_floor=0.0) == base
    assert oracle.ccm_unit(s, 1, 0, 3, 1, 120, 0, 7, theiler=5) != base
    assert oracle.ccm_unit(s, 1, 0, 3, 1, 120, 0, 7, weight_floor=0.2) != base


def test_option_arguments_are_checked():
    s = I.logistic_pair(100)
    with pytest.raises(ValueError):      # L < E + 2 + 2W
        oracle.ccm_unit(s, 1, 0, 2, 1, 9, 0, 1, theiler=3)
    oracle.ccm_unit(s, 1, 0, 2, 1, 10, 0, 1, theiler=3)
    with pytest.raises(ValueError):
        oracle.ccm_unit(s, 1, 0, 2, 1, 50, 0, 1, theiler=-1)
    with pytest.raises(ValueError):
        oracle.ccm_unit(s, 1, 0, 2, 1, 50, 0, 1, weight_floor=-0.5)
    with pytest.raises(ValueError):
        oracle.ccm_unit(s, 1, 0, 2, 1, 50, 0, 1, weight_floor=float("nan"))
