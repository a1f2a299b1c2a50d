"""Pins of the CPU oracle against things other than itself (no GPU needed).

The paper prints no worked example and no skill values, so every pin here is
fixed by mathematics, a library routine, brute force or the known dynamics of
the coupled logistic map that the method's source (Sugihara et al. 2012, cited
in the paper's Sect. 2.1) studies:

* Philox4x64-10 against numpy's independent implementation;
* libraries against a numpy re-derivation of the random-key selection;
* neighbour lists against pure-Python brute force (exact FP32 fused
  multiply-add emulation with rationals, and plain FP64);
* simplex weights on a hand-worked 10-point example (tests/golden);
* predictions against pure-Python brute force at E > 1, tau > 1;
* rho against numpy.corrcoef;
* invariances (library order, power-of-two scaling, affine target map);
* special cases (L = N_m) and convergence of rho with L.
"""

from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1905_00565_gb300 import inputs as I

MASK64 = (1 << 64) - 1
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox ----
def numpy_philox_block(ctr, key):
    """Philox4x64-10 block at counter ``ctr`` from numpy's bit generator.

    numpy increments its 256-bit counter (word 0 least significant) before it
    draws a block, so the block at ``ctr`` is the first block drawn from a
    generator whose counter is ``ctr - 1``.
    """
    c = sum(int(w) << (64 * q) for q, w in enumerate(ctr))
    c = (c - 1) % (1 << 256)
    words = np.array([(c >> (64 * q)) & MASK64 for q in range(4)], dtype=np.uint64)
    g = np.random.Philox(counter=words, key=np.array(key, dtype=np.uint64))
    return g.random_raw(4)


@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([1, 2, 3, 4], [5, 6]),
    ([MASK64, MASK64, MASK64, MASK64], [MASK64, MASK64]),
    ([0, 1, 0, 0], [20190501, 0]),
    ([123456789, 7, 9000, (63 << 16) | (10 << 8) | 4], [20190503, 0]),
])
def test_philox_matches_numpy(ctr, key):
    got = oracle.philox4x64_10(ctr, key)
    want = numpy_philox_block(ctr, key)
    assert [int(x) for x in got] == [int(x) for x in want]


def test_philox_matches_numpy_random():
    rng = np.random.default_rng(7)
    for _ in range(50):
        ctr = [int(x) for x in rng.integers(0, 2**63, size=4, dtype=np.int64)]
        key = [int(x) for x in rng.integers(0, 2**63, size=2, dtype=np.int64)]
        assert [int(x) for x in oracle.philox4x64_10(ctr, key)] == \
               [int(x) for x in numpy_philox_block(ctr, key)]


# --------------------------------------------------------------- library ----
def numpy_library(n_m, L, j, E, tau, k, seed):
    """Random-key selection restated with numpy's Philox and Python sorting:
    point m's key is 32-bit half m mod 8 (high half of word 0 first) of the
    block at counter m // 8, then m."""
    keys = []
    for m in range(n_m):
        block = numpy_philox_block([m // 8, k, L, (j << 16) | (E << 8) | tau], [seed, 0])
        halves = [h for w in block for h in (int(w) >> 32, int(w) & 0xFFFFFFFF)]
        keys.append((halves[m % 8] << 32) | m)
    keys.sort()
    return np.array(sorted(x & 0xFFFFFFFF for x in keys[:L]), dtype=np.int32)


@pytest.mark.parametrize("n_m,L,j,E,tau,k,seed", [
    (40, 5, 0, 1, 1, 0, 1),
    (97, 50, 1, 2, 1, 3, 20190502),
    (200, 199, 63, 10, 4, 249, 20190503),
    (64, 64, 5, 3, 2, 1, 9),
])
def test_library_matches_numpy_rederivation(n_m, L, j, E, tau, k, seed):
    got = oracle.library(n_m, L, j, E, tau, k, seed)
    assert np.array_equal(got, numpy_library(n_m, L, j, E, tau, k, seed))


def test_library_properties():
    for (n_m, L) in [(10, 3), (500, 100), (1000, 999), (37, 37)]:
        for k in range(5):
            lib = oracle.library(n_m, L, 1, 2, 1, k, 11)
            assert len(lib) == L
            assert np.all(np.diff(lib) > 0)          # ascending, hence distinct
            assert lib[0] >= 0 and lib[-1] < n_m
    # L = N_m: the library is the whole manifold
    assert np.array_equal(oracle.library(73, 73, 0, 4, 3, 17, 5), np.arange(73))


def test_library_inclusion_is_uniform():
    """Each point is drawn with probability L/N_m (binomial bound over 2000 draws)."""
    n_m, L, R = 50, 10, 2000
    counts = np.zeros(n_m)
    for k in range(R):
        counts[oracle.library(n_m, L, 0, 1, 1, k, 99)] += 1
    p = L / n_m
    sd = math.sqrt(R * p * (1 - p))
    assert np.all(np.abs(counts - R * p) < 5 * sd)
    # libraries of different L (and different k) are drawn independently
    a = oracle.library(1000, 100, 0, 2, 1, 0, 3)
    b = oracle.library(1000, 101, 0, 2, 1, 0, 3)
    assert len(np.intersect1d(a, b)) < 40


# ----------------------------------------------------- brute-force kNN ------
def _round_to_f32(v: Fraction) -> np.float32:
    """Round an exact rational to the nearest float32, ties to even."""
    f = np.float32(float(v))
    cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]

    def key(c):
        return (abs(Fraction(float(c)) - v), int(np.array(c, np.float32).view(np.uint32)) & 1)

    return min(cands, key=key)


def _fma32(a, b, c):
    return _round_to_f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def _coords(s, E, tau, m):
    return [s[m + (E - 1) * tau - e * tau] for e in range(E)]


def _sqdist32(s, E, tau, a, b, reverse=False, fused=True):
    """FP32 squared distance: first term a rounded product, then one rounding per
    fused multiply-add, coordinates taken from e=0 (the value at t) upward.  The
    ``reverse``/``fused=False`` variants are the plausible wrong sequences."""
    ca, cb = _coords(s, E, tau, a), _coords(s, E, tau, b)
    order = list(range(E))[::-1] if reverse else list(range(E))
    diff = np.float32(ca[order[0]]) - np.float32(cb[order[0]])
    acc = np.float32(diff * diff)
    for e in order[1:]:
        diff = np.float32(ca[e]) - np.float32(cb[e])
        acc = _fma32(diff, diff, acc) if fused else np.float32(acc + np.float32(diff * diff))
    return float(acc)


def _sqdist64(s, E, tau, a, b):
    ca, cb = _coords(s, E, tau, a), _coords(s, E, tau, b)
    acc = 0.0
    for e in range(E):
        d = float(ca[e]) - float(cb[e])
        acc = acc + d * d
    return acc


def brute_neighbours(s, E, tau, lib, fp64, **variant):
    n_m = len(s) - (E - 1) * tau
    out = []
    for m in range(n_m):
        if fp64:
            cand = sorted((_sqdist64(s, E, tau, m, int(l)), int(l)) for l in lib if int(l) != m)
        else:
            cand = sorted((_sqdist32(s, E, tau, m, int(l), **variant), int(l))
                          for l in lib if int(l) != m)
        out.append([l for _, l in cand[:E + 1]])
    return np.array(out, dtype=np.int32)


def _tiny_series(kind, n, rng):
    if kind == "uniform":
        return rng.random(n).astype(np.float32)
    if kind == "integers":                       # many exact ties
        return rng.integers(0, 5, size=n).astype(np.float32)
    x = I.logistic_pair(n + 17)[1][17:]
    return np.ascontiguousarray(x)


@pytest.mark.parametrize("kind", ["uniform", "integers", "logistic"])
@pytest.mark.parametrize("fp64", [False, True])
def test_neighbours_match_brute_force(kind, fp64):
    rng = np.random.default_rng(hash((kind, fp64)) & 0xFFFF)
    for E in range(1, 5):
        for tau in range(1, 4):
            n = int(rng.integers(E * tau + 8, 41))
            s = _tiny_series(kind, n, rng)
            n_m = n - (E - 1) * tau
            for L in sorted({E + 2, (E + 2 + n_m) // 2, n_m}):
                lib = np.sort(rng.choice(n_m, size=L, replace=False)).astype(np.int32)
                got = oracle.neighbours(s, E, tau, lib, select_fp64=fp64)
                want = brute_neighbours(s, E, tau, lib, fp64)
                assert np.array_equal(got, want), (kind, E, tau, L)


def mirrored_near_tie_series(rng):
    """E=2, tau=1 series whose query 0 has two candidates with mirrored coordinate
    differences (d1, d2) and (d2, d1): equal in exact arithmetic, so the FP32
    rounding sequence alone decides which one is the 3rd (= E+1-th) neighbour.
    Two closer points come first; filler values keep every other point far."""
    q0, q1 = 0.5, 0.25
    d1, d2 = (float(np.float32(x)) for x in rng.uniform(0.01, 0.02, size=2))
    F = 1000.0
    s = [q0, q1, F,
         q0 - d2, q1 - d1, F,          # point 3: coordinates (s[4], s[3]) -> diffs (d1, d2)
         q0 - d1, q1 - d2, F,          # point 6: diffs (d2, d1)
         q0 + 1e-3, q1 + 1e-3, F,      # point 9: clearly closer
         q0 - 2e-3, q1 + 1e-3, F, F]   # point 12: clearly closer
    return np.array(s, dtype=np.float32)


def test_fp32_rounding_sequence_is_pinned():
    """The FP32 selection follows one rounding sequence (coordinates from the value
    at t backwards, fused multiply-add).  On mirrored near ties the reversed order
    and the unfused sum pick differently; the oracle must pick as specified."""
    rng = np.random.default_rng(11)
    lib = None
    hits = {"reverse": 0, "unfused": 0}
    for _ in range(200):
        s = mirrored_near_tie_series(rng)
        n_m = len(s) - 1
        lib = np.arange(n_m, dtype=np.int32)
        want = brute_neighbours(s, 2, 1, lib, False)[0]
        got = oracle.neighbours(s, 2, 1, lib)[0]
        assert list(got) == list(want)
        if list(brute_neighbours(s, 2, 1, lib, False, reverse=True)[0]) != list(want):
            hits["reverse"] += 1
        if list(brute_neighbours(s, 2, 1, lib, False, fused=False)[0]) != list(want):
            hits["unfused"] += 1
    # the construction really discriminates between the sequences
    assert hits["reverse"] >= 3 and hits["unfused"] >= 3, hits


def test_neighbours_e1_are_a_window_in_value_order():
    """E=1: the E+1 nearest values form a contiguous run of the sorted library."""
    rng = np.random.default_rng(3)
    s = rng.random(60).astype(np.float32)
    lib = np.sort(rng.choice(60, size=30, replace=False)).astype(np.int32)
    nbr = oracle.neighbours(s, 1, 1, lib)
    for m in range(60):
        others = [int(l) for l in lib if l != m]
        order = sorted(others, key=lambda l: (float(s[l]), l))
        pos = sorted(order.index(int(l)) for l in nbr[m])
        assert pos == list(range(pos[0], pos[0] + 2))
        # and nothing outside the run is strictly closer than the run's farthest
        far = max(abs(float(s[l]) - float(s[m])) for l in nbr[m])
        assert all(abs(float(s[l]) - float(s[m])) >= far for l in others if l not in nbr[m])


# ------------------------------------------------------ hand-worked example --
def _read_golden():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "simplex_10pt.txt"))
            if ln.strip() and not ln.startswith("#")]
    Y = np.array([float(v) for v in rows[0][1:]], np.float32)
    X = np.array([float(v) for v in rows[1][1:]], np.float32)
    table = [(int(r[0]), int(r[1]), int(r[2]), float(r[3]), float(r[4])) for r in rows[2:]]
    return Y, X, table


def test_simplex_hand_worked_example():
    Y, X, table = _read_golden()
    lib = np.arange(10, dtype=np.int32)
    nbr = oracle.neighbours(Y, 1, 1, lib)
    xhat = oracle.predict(Y, X, 1, 1, nbr)
    for m, n1, n2, d1, d2 in table:
        assert list(nbr[m]) == [n1, n2]
        if d1 > 0:
            g = math.exp(-(d2 - d1) / d1)
            want = (float(X[n1]) + float(X[n2]) * g) / (1.0 + g)
        else:
            want = float(X[n1])
        assert xhat[m] == pytest.approx(want, rel=1e-14, abs=0)


# ------------------------------------------- brute-force prediction, E > 1 --
def brute_predict(ls, ts, E, tau, nbr):
    out = []
    for m, row in enumerate(nbr):
        d = [math.sqrt(_sqdist64(ls, E, tau, m, int(l))) for l in row]
        d1 = min(d)
        u = [math.exp(-x / d1) if d1 > 0 else (1.0 if x == 0 else 0.0) for x in d]
        out.append(sum(ui * float(ts[int(l) + (E - 1) * tau]) for ui, l in zip(u, row)) / sum(u))
    return np.array(out)


def test_predictions_match_brute_force():
    rng = np.random.default_rng(5)
    s = I.logistic_pair(80)
    for E, tau in [(2, 1), (3, 2), (4, 3), (1, 4)]:
        n_m = 80 - (E - 1) * tau
        lib = np.sort(rng.choice(n_m, size=n_m // 2, replace=False)).astype(np.int32)
        nbr = oracle.neighbours(s[1], E, tau, lib)
        got = oracle.predict(s[1], s[0], E, tau, nbr)
        want = brute_predict(s[1], s[0], E, tau, nbr)
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=0)
        # skill: the observed target is aligned at t_m = m + (E-1)tau
        obs = s[0][(E - 1) * tau:].astype(np.float64)
        assert oracle.skill(s[0], E, tau, got) == pytest.approx(np.corrcoef(obs, got)[0, 1],
                                                                abs=1e-12)


# ------------------------------------------------------------------ rho -----
def test_pearson_matches_numpy_corrcoef():
    rng = np.random.default_rng(1)
    for n in [2, 3, 10, 1000, 10007]:
        x = rng.random(n) * 3 + 5
        y = 0.3 * x + rng.random(n)
        assert oracle.pearson(x, y) == pytest.approx(np.corrcoef(x, y)[0, 1], abs=1e-12)
    assert math.isnan(oracle.pearson(np.ones(5), np.arange(5.0)))


def test_unit_rho_is_corrcoef_of_its_predictions():
    p = I.plain_ccm_problem()
    rho, lib, nbr, xh = oracle.ccm_unit(p.series, 1, 0, 2, 1, 200, 3, p.seed, keep=True)
    obs = p.series[0][1:].astype(np.float64)
    assert rho == pytest.approx(np.corrcoef(obs, xh)[0, 1], abs=1e-12)
    assert np.array_equal(lib, oracle.library(999, 200, 1, 2, 1, 3, p.seed))
    assert np.array_equal(nbr, oracle.neighbours(p.series[1], 2, 1, lib))


# ------------------------------------------------------------ invariants ----
def test_library_order_does_not_matter():
    rng = np.random.default_rng(2)
    s = I.logistic_pair(300)[1]
    lib = np.sort(rng.choice(299, size=120, replace=False)).astype(np.int32)
    a = oracle.neighbours(s, 2, 1, lib)
    b = oracle.neighbours(s, 2, 1, rng.permutation(lib).astype(np.int32))
    assert np.array_equal(a, b)


def test_power_of_two_scaling_is_exact():
    s = I.logistic_pair(300)
    lib = oracle.library(297, 150, 1, 3, 1, 0, 4)
    nb = oracle.neighbours(s[1], 3, 1, lib)
    xh = oracle.predict(s[1], s[0], 3, 1, nb)
    for k in (-3, 5):
        sc = (s[1] * np.float32(2.0 ** k)).astype(np.float32)
        nb2 = oracle.neighbours(sc, 3, 1, lib)
        assert np.array_equal(nb, nb2)
        assert np.array_equal(xh, oracle.predict(sc, s[0], 3, 1, nb2))


def test_affine_target_map_keeps_rho():
    s = I.logistic_pair(400)
    rho = oracle.ccm_unit(s, 1, 0, 2, 1, 300, 0, 1)
    t = s.copy()
    t[0] = (2.5 * s[0].astype(np.float64) - 1.0).astype(np.float32)
    rho2 = oracle.ccm_unit(t, 1, 0, 2, 1, 300, 0, 1)
    assert rho2 == pytest.approx(rho, abs=1e-6)   # FP32 rounding of the mapped target


def test_full_library_realizations_are_identical():
    s = I.logistic_pair(200)
    n_m = 200 - 2
    rhos = [oracle.ccm_unit(s, 1, 0, 3, 1, n_m, k, 8) for k in range(4)]
    assert all(r == rhos[0] for r in rhos)


def test_fp32_selection_differs_from_fp64_only_at_near_ties():
    """FP32 and FP64 selections agree except where the FP64 gap is < 1e-6 relative."""
    s = I.logistic_pair(600)
    for E, tau in [(1, 1), (2, 1), (5, 2), (10, 1)]:
        n_m = 600 - (E - 1) * tau
        for k in range(3):
            lib = oracle.library(n_m, 300, 1, E, tau, k, 12)
            a = oracle.neighbours(s[1], E, tau, lib, select_fp64=False)
            b = oracle.neighbours(s[1], E, tau, lib, select_fp64=True)
            rows = np.nonzero(np.any(np.sort(a, 1) != np.sort(b, 1), axis=1))[0]
            for m in rows:
                d = sorted(math.sqrt(_sqdist64(s[1], E, tau, int(m), int(l)))
                           for l in lib if l != m)
                assert (d[E + 1] - d[E]) <= 1e-6 * d[E + 1]
            if len(rows):
                assert np.all(oracle.query_margin(s[1], E, tau, lib, rows) < 1e-6)


def brute_margin(s, E, tau, lib, m, theiler=0):
    """Pure-Python relative FP64 gap between the (E+1)-th and (E+2)-th nearest
    candidate distances of query m (inf with only E+1 candidates, 0 at d_b = 0)."""
    d2 = sorted(_sqdist64(s, E, tau, m, int(l)) for l in lib if abs(int(l) - m) > theiler)
    if len(d2) < E + 2:
        return math.inf
    da, db = math.sqrt(d2[E]), math.sqrt(d2[E + 1])
    return (db - da) / db if db > 0.0 else 0.0


@pytest.mark.parametrize("kind", ["uniform", "integers", "logistic"])
def test_query_margin_matches_brute_force(kind):
    rng = np.random.default_rng(hash(kind) & 0xFFFF)
    for E in range(1, 5):
        for tau in range(1, 4):
            n = int(rng.integers(E * tau + 12, 41))
            s = _tiny_series(kind, n, rng)
            n_m = n - (E - 1) * tau
            for W in (0, 2):
                for L in sorted({E + 2 + 2 * W, n_m}):
                    lib = np.sort(rng.choice(n_m, size=L, replace=False)).astype(np.int32)
                    q = np.arange(n_m)
                    got = oracle.query_margin(s, E, tau, lib, q, theiler=W)
                    want = [brute_margin(s, E, tau, lib, int(m), W) for m in q]
                    assert np.array_equal(got, np.array(want)), (kind, E, tau, L, W)


def test_query_margin_closed_forms():
    """E = 1 on the values 0, 1, 3, 6, 10, 15: from point 0 the candidates lie at
    1, 3, 6, 10, 15, so the 2nd and 3rd nearest give (6 - 3)/6 = 1/2; from point 2
    (value 3) they lie at 2, 3, 3, 7, 12: (3 - 3)/3 = 0 (an exact tie).  With only
    E+1 = 2 candidates the set cannot be contested: inf.  A duplicate-heavy series
    gives d_b = 0: 0."""
    s = np.array([0, 1, 3, 6, 10, 15], np.float32)
    lib = np.arange(6, dtype=np.int32)
    g = oracle.query_margin(s, 1, 1, lib, [0, 2])
    assert g[0] == 0.5 and g[1] == 0.0
    assert oracle.query_margin(s, 1, 1, np.array([0, 1, 2], np.int32), [0])[0] == math.inf
    z = np.array([1, 1, 1, 1, 5], np.float32)
    assert oracle.query_margin(z, 1, 1, np.arange(5, dtype=np.int32), [0])[0] == 0.0
    with pytest.raises(ValueError):
        oracle.query_margin(s, 1, 1, lib, [6])


# --------------------------------------------------------------- dynamics ---
def test_convergence_of_the_coupled_logistic_map():
    """Strongly driven direction: rho rises with L, exceeds 0.8 at L=800, and beats
    the weakly driven direction at every L >= 200 (Sugihara et al. 2012 system)."""
    p = I.plain_ccm_problem()
    rho = oracle.ccm(p.series, p.pairs, p.E, p.tau, p.L, p.r, p.seed)
    mean = rho.mean(axis=-1)[:, 0, 0, :]          # [pair][L]
    strong, weak = mean[0], mean[1]               # (lib M_Y -> X), (lib M_X -> Y)
    assert np.all(np.diff(strong) > 0)
    assert strong[-1] > 0.8
    assert np.all(strong[2:] > weak[2:])
    assert np.all(np.isfinite(rho))


def test_query_subset_matches_full_run():
    s = I.logistic_pair(500)
    lib = oracle.library(497, 200, 1, 4, 1, 2, 3)
    nbr = oracle.neighbours(s[1], 4, 1, lib)
    xh = oracle.predict(s[1], s[0], 4, 1, nbr)
    q = np.array([0, 7, 250, 496])
    nb2, xh2 = oracle.query_subset(s[1], s[0], 4, 1, lib, q)
    assert np.array_equal(nb2, nbr[q])
    assert np.array_equal(xh2, xh[q])
