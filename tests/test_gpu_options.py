"""The two optional CCM variants on the GPU (exclusion window W, weight floor f;
not in the paper, both off by default) against the oracle, the plain
comparator, the distance-indexing-table path and the serving path (needs a
GB300)."""

from __future__ import annotations

import time

import numpy as np
import pytest

from paper_1905_00565_gb300 import inputs as I
from tests.ccm_check import check_units, run_detailed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccm():
    from paper_1905_00565_gb300 import ccm as c
    return c


def small(theiler, floor, n=1200, r=3):
    return I.Problem(series=I.logistic_pair(n), pairs=I.BOTH_DIRECTIONS.copy(),
                     E=np.array([1, 3, 6], np.int32), tau=np.array([1, 2], np.int32),
                     L=np.array([60, 400, 1100], np.int64), r=r, seed=17,
                     name=f"opts-W{theiler}-f{floor}", theiler=theiler, weight_floor=floor)


@pytest.mark.parametrize("theiler,floor", [(3, 0.0), (17, 0.0), (0, 1e-3), (5, 0.2)])
def test_options_match_oracle_and_plain(ccm, theiler, floor):
    p = small(theiler, floor)
    ctx = ccm.ccm_context_create(0)
    try:
        rho, lib, nbr, xh = run_detailed(ccm, ctx, p)
        plan = ccm.plan_problem(ctx, p)
        try:
            rho_plain = np.zeros_like(rho)
            ccm.ccm_run_plain(plan, p.series, rho_plain)
        finally:
            ccm.ccm_plan_destroy(plan)
    finally:
        ccm.ccm_context_destroy(ctx)
    check_units(p, rho, lib, nbr, xh)
    np.testing.assert_allclose(rho, rho_plain, rtol=0, atol=1e-12)
    # the window really excludes: no neighbour within W of its query
    if theiler:
        off = 0
        for E in p.E:
            for tau in p.tau:
                n_m = p.n - (int(E) - 1) * int(tau)
                for _ in range(len(p.L) * p.r):
                    rows = nbr[off:off + n_m * (E + 1)].reshape(n_m, E + 1)
                    assert np.all(np.abs(rows - np.arange(n_m)[:, None]) > theiler)
                    off += n_m * (E + 1)


def test_options_change_results(ccm):
    ctx = ccm.ccm_context_create(0)
    try:
        out = {}
        for key in [(0, 0.0), (9, 0.0), (0, 0.3)]:
            p = small(*key, r=2)
            plan = ccm.plan_problem(ctx, p)
            try:
                out[key] = np.zeros(ccm.rho_shape(p))
                ccm.ccm_run(plan, p.series, out[key])
            finally:
                ccm.ccm_plan_destroy(plan)
    finally:
        ccm.ccm_context_destroy(ctx)
    assert not np.array_equal(out[(0, 0.0)], out[(9, 0.0)])
    assert not np.array_equal(out[(0, 0.0)], out[(0, 0.3)])


def test_window_with_tables_equals_brute_force(ccm):
    base = I.sweep_problem()
    s = np.ascontiguousarray(base.series[:, :4000])
    p = I.Problem(series=s, pairs=I.BOTH_DIRECTIONS.copy(), E=np.array([2, 5], np.int32),
                  tau=np.array([1], np.int32), L=np.array([900, 3500], np.int64), r=12,
                  seed=base.seed, name="window-table", theiler=12, weight_floor=1e-4)
    ctx = ccm.ccm_context_create(0)
    try:
        plan = ccm.plan_problem(ctx, p)
        try:
            assert ccm.ccm_plan_get_info(plan)["table_bytes"] > 0
        finally:
            ccm.ccm_plan_destroy(plan)
        r0, l0, n0, x0 = run_detailed(ccm, ctx, p, ccm.CCM_NO_TABLE)
        r1, l1, n1, x1 = run_detailed(ccm, ctx, p, 0)
    finally:
        ccm.ccm_context_destroy(ctx)
    assert np.array_equal(n0, n1) and np.array_equal(x0, x1) and np.array_equal(r0, r1)
    check_units(p, r1, l1, n1, x1, which={0, 13, 30, 47})


def test_served_job_with_options_equals_run_alone(ccm):
    p = small(4, 0.01, r=4)
    q = small(0, 0.0, r=4)
    ctx = ccm.ccm_context_create(0)
    try:
        alone = {}
        for name, prob in [("opt", p), ("plain", q)]:
            plan = ccm.plan_problem(ctx, prob)
            try:
                alone[name] = np.zeros(ccm.rho_shape(prob))
                ccm.ccm_run(plan, prob.series, alone[name])
            finally:
                ccm.ccm_plan_destroy(plan)
        t1 = ccm.ccm_submit(ctx, p.series, p.pairs, p.E, p.tau, p.L, p.r, p.seed,
                            theiler=p.theiler, weight_floor=p.weight_floor)
        t2 = ccm.ccm_submit(ctx, q.series, q.pairs, q.E, q.tau, q.L, q.r, q.seed)
        for t, name, prob in [(t1, "opt", p), (t2, "plain", q)]:
            rho = np.zeros(ccm.rho_shape(prob))
            t0 = time.time()
            while ccm.ccm_poll(ctx, t, rho, 200) != ccm.CCM_OK:
                assert time.time() - t0 < 120
            assert np.max(np.abs(rho - alone[name])) <= 1e-12
    finally:
        ccm.ccm_context_destroy(ctx)


def test_invalid_options_are_refused(ccm):
    ctx = ccm.ccm_context_create(0)
    try:
        bad = [small(-1, 0.0), small(0, -0.5), small(0, float("nan")), small(30, 0.0)]
        for p in bad:     # W = 30 needs L >= E + 2 + 60 > 60
            with pytest.raises(ccm.CCMError) as ei:
                ccm.plan_problem(ctx, p)
            assert ei.value.status == ccm.CCM_EINVAL
    finally:
        ccm.ccm_context_destroy(ctx)


def test_completion_count_range_is_checked(ccm):
    """A realization completes after (query tiles) x (targets of its library
    variable) reductions, counted in 32 bits: a problem reaching 2^31 is
    refused before anything is allocated (only the series shape is given)."""
    n = 2**31 - 1                                # ceil(n/256) = 8388608 tiles
    many = np.array([[0, i] for i in range(1, 257)], np.int32)   # 256 targets of j = 0
    ctx = ccm.ccm_context_create(0)
    try:
        with pytest.raises(ccm.CCMError) as ei:
            ccm.ccm_plan(ctx, (257, n), many, [2], [1], [10], 1, 1)
        assert ei.value.status == ccm.CCM_EINVAL
        assert "2^31" in str(ei.value)
    finally:
        ccm.ccm_context_destroy(ctx)
