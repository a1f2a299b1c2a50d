"""Distance indexing tables (paper Sect. 3.2; on by default) on the GPU.

A realization that reads its neighbours from the table must give exactly what
the brute-force search gives (same neighbour lists, same bits of rho): the
table row is the whole manifold sorted by (FP32 squared distance, index), and
restricting it to the library keeps that order.  Checked against the
brute-force path bit for bit, against the oracle, on tie-heavy integer series,
with the fallback path forced by a tiny safety factor, and on the long series.
"""

from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from paper_1905_00565_gb300 import inputs as I
from tests.ccm_check import XHAT_RTOL, check_units, run_detailed, split, xhat_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccm():
    from paper_1905_00565_gb300 import ccm as c
    return c


def both_paths(ccm, ctx, p):
    """(brute force everywhere, default with tables)"""
    a = run_detailed(ccm, ctx, p, ccm.CCM_NO_TABLE)
    b = run_detailed(ccm, ctx, p, 0)
    return a, b


def uses_table(ccm, ctx, p):
    plan = ccm.plan_problem(ctx, p)
    try:
        return ccm.ccm_plan_get_info(plan)["table_bytes"] > 0
    finally:
        ccm.ccm_plan_destroy(plan)


def test_table_equals_brute_force_and_oracle(ccm):
    base = I.sweep_problem()
    s = np.ascontiguousarray(base.series[:, :3000])
    p = I.Problem(series=s, pairs=I.BOTH_DIRECTIONS.copy(), E=np.array([1, 2, 5, 10], np.int32),
                  tau=np.array([1, 3], np.int32), L=np.array([150, 300, 1200, 2900], np.int64),
                  r=6, seed=base.seed, name="table-cells")
    ctx = ccm.ccm_context_create(0)
    try:
        assert uses_table(ccm, ctx, p)
        (r0, l0, n0, x0), (r1, l1, n1, x1) = both_paths(ccm, ctx, p)
    finally:
        ccm.ccm_context_destroy(ctx)
    assert np.array_equal(l0, l1) and np.array_equal(n0, n1)
    assert np.array_equal(x0, x1) and np.array_equal(r0, r1)
    rng = np.random.default_rng(3)
    check_units(p, r1, l1, n1, x1, which=set(int(u) for u in rng.choice(r1.size, 12, replace=False)))


def rho_only(ccm, ctx, p, flags):
    plan = ccm.plan_problem(ctx, p, flags)
    try:
        rho = np.zeros(ccm.rho_shape(p))
        ccm.ccm_run(plan, p.series, rho)
    finally:
        ccm.ccm_plan_destroy(plan)
    return rho


def test_table_target_values_match_brute_force(ccm):
    """Without neighbour lists requested, a table of a variable with one target
    holds (distance, target value) pairs and the scan reads the target's values
    from it; with several targets per variable it gathers them.  Either way rho
    is bit-identical to brute force, and to the run that also returns the
    neighbour lists (which reads the indices)."""
    base = I.sweep_problem()
    s = np.ascontiguousarray(base.series[:, :3000])
    one = I.Problem(series=s, pairs=I.BOTH_DIRECTIONS.copy(), E=np.array([2, 7], np.int32),
                    tau=np.array([1, 2], np.int32), L=np.array([300, 1400, 2900], np.int64),
                    r=9, seed=base.seed, name="one-target")
    s3 = np.ascontiguousarray(np.vstack([s, s[:1] * 0.5 + s[1:] * 0.5]))
    many = I.Problem(series=s3, pairs=np.array([[0, 1], [0, 2], [1, 0], [2, 1]], np.int32),
                     E=np.array([3], np.int32), tau=np.array([1], np.int32),
                     L=np.array([400, 1500, 2900], np.int64), r=9, seed=base.seed,
                     name="two-targets")
    ctx = ccm.ccm_context_create(0)
    try:
        for p in (one, many):
            assert uses_table(ccm, ctx, p)
            brute = rho_only(ccm, ctx, p, ccm.CCM_NO_TABLE)
            table = rho_only(ccm, ctx, p, 0)
            detailed = run_detailed(ccm, ctx, p, 0)[0]
            np.testing.assert_array_equal(table, brute)
            np.testing.assert_array_equal(table, detailed)
    finally:
        ccm.ccm_context_destroy(ctx)


def test_table_with_exact_ties_and_full_library(ccm):
    rng = np.random.default_rng(8)
    ints = rng.integers(0, 6, size=(2, 2500)).astype(np.float32)
    p = I.Problem(series=ints, pairs=I.BOTH_DIRECTIONS.copy(), E=np.array([1, 2, 3], np.int32),
                  tau=np.array([1], np.int32), L=np.array([300, 2498], np.int64), r=10, seed=4,
                  name="ties")
    ctx = ccm.ccm_context_create(0)
    try:
        assert uses_table(ccm, ctx, p)
        (r0, l0, n0, x0), (r1, l1, n1, x1) = both_paths(ccm, ctx, p)
    finally:
        ccm.ccm_context_destroy(ctx)
    assert np.array_equal(n0, n1) and np.array_equal(x0, x1)
    np.testing.assert_array_equal(r0, r1)
    check_units(p, r1, l1, n1, x1, which={0, 5, 11, 37, 63})


def test_table_fallback_path(ccm, monkeypatch):
    """A tiny safety factor leaves many queries with fewer than E+1 library
    members among their R table entries; they scan their library instead."""
    monkeypatch.setenv("CCM_TABLE_SAFETY", "0.05")
    base = I.sweep_problem()
    s = np.ascontiguousarray(base.series[:, :4000])
    p = I.Problem(series=s, pairs=I.BOTH_DIRECTIONS.copy(), E=np.array([3, 8], np.int32),
                  tau=np.array([2], np.int32), L=np.array([400, 3000], np.int64), r=12,
                  seed=base.seed, name="fallback")
    ctx = ccm.ccm_context_create(0)
    try:
        assert uses_table(ccm, ctx, p)
        (r0, l0, n0, x0), (r1, l1, n1, x1) = both_paths(ccm, ctx, p)
    finally:
        ccm.ccm_context_destroy(ctx)
    assert np.array_equal(n0, n1) and np.array_equal(r0, r1)


def test_table_fallback_small_e_regression(ccm, monkeypatch):
    """E = 2, tau = 3 on the full 10^4-point series with short table rows: at
    L = 850 some queries meet fewer than E+1 library members among their
    table entries and scan their library; the scan must keep the whole sorted
    (distance, index) list."""
    monkeypatch.setenv("CCM_TABLE_SAFETY", "0.05")
    base = I.sweep_problem()
    p = I.Problem(series=base.series, pairs=np.array([[1, 0]], np.int32),
                  E=np.array([2], np.int32), tau=np.array([3], np.int32),
                  L=np.array([850, 9000], np.int64), r=29, seed=base.seed, name="fallback-e2")
    ctx = ccm.ccm_context_create(0)
    try:
        assert uses_table(ccm, ctx, p)
        (r0, l0, n0, x0), (r1, l1, n1, x1) = both_paths(ccm, ctx, p)
    finally:
        ccm.ccm_context_destroy(ctx)
    assert np.array_equal(n0, n1) and np.array_equal(r0, r1)
    check_units(p, r1, l1, n1, x1, which={0, 3, 30, 57})


def test_table_on_the_long_series_sampled(ccm):
    base = I.long_series_problem()
    p = I.Problem(series=base.series, pairs=base.pairs, E=np.array([4], np.int32),
                  tau=np.array([1], np.int32), L=np.array([5000, 50000], np.int64), r=16,
                  seed=base.seed, name="long-table")
    ctx = ccm.ccm_context_create(0)
    try:
        assert uses_table(ccm, ctx, p)
        rho, lib, nbr, xh = run_detailed(ccm, ctx, p, 0)
        rb, *_ = run_detailed(ccm, ctx, p, ccm.CCM_NO_TABLE)
    finally:
        ccm.ccm_context_destroy(ctx)
    np.testing.assert_array_equal(rho, rb)
    rng = np.random.default_rng(6)
    for (u, j, i, E, tau, L, k, n_m, l_g, n_g, x_g) in split(p, lib, nbr, xh):
        if u not in (0, 7, 16, 31):
            continue
        q = np.sort(rng.choice(n_m, size=200, replace=False))
        nb_o, xh_o = oracle.query_subset(p.series[j], p.series[i], E, tau, l_g, q)
        assert np.array_equal(n_g[q], nb_o)
        assert xhat_rel_err(x_g[q], xh_o, p.series[i]) <= XHAT_RTOL
