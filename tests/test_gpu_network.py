"""Network-wide CCM (64 coupled logistic variables, all ordered pairs) with
neighbour reuse: one library and one neighbour search per (library variable,
E, tau, L, k) serve all 63 targets (needs a GB300).

Checks: sampled realizations against the oracle (libraries and neighbours
bit-exact, predictions, rho); every rho against the plain comparator, which
cross-maps each target separately; and the full 4032-pair sweep's rho on
sampled realizations.
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1905_00565_gb300 import inputs as I
from tests.ccm_check import RHO_TOL, check_units, run_detailed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def net():
    return I.network_problem()


def test_network_subset_reuse_matches_oracle_and_plain(net):
    from paper_1905_00565_gb300 import ccm
    pairs = np.array([[j, i] for j in (3, 40) for i in range(64) if i != j], np.int32)
    p = I.Problem(series=net.series, pairs=pairs, E=np.array([2, 4], np.int32),
                  tau=np.array([1], np.int32), L=np.array([100, 4500], np.int64), r=2,
                  seed=net.seed, name="network-subset")
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
    np.testing.assert_allclose(rho, rho_plain, rtol=0, atol=1e-12)
    rng = np.random.default_rng(5)
    which = set(int(x) for x in rng.choice(rho.size, size=10, replace=False))
    check_units(p, rho, lib, nbr, xh, which=which)


def test_full_network_sweep_sampled(net):
    from paper_1905_00565_gb300 import ccm
    p = net
    ctx = ccm.ccm_context_create(0)
    try:
        plan = ccm.plan_problem(ctx, p)
        try:
            info = ccm.ccm_plan_get_info(plan)
            assert info["n_units"] == 4032 * 3 * 8 * 250
            rho = np.zeros(ccm.rho_shape(p))
            ccm.ccm_run(plan, p.series, rho)
        finally:
            ccm.ccm_plan_destroy(plan)
    finally:
        ccm.ccm_context_destroy(ctx)
    assert np.all(np.isfinite(rho)) and np.all(np.abs(rho) <= 1.0)
    rng = np.random.default_rng(9)
    for _ in range(6):
        pi, e, l, k = (int(rng.integers(0, 4032)), int(rng.integers(0, 3)),
                       int(rng.integers(0, 8)), int(rng.integers(0, 250)))
        j, i = (int(x) for x in p.pairs[pi])
        r_o = oracle.ccm_unit(p.series, j, i, int(p.E[e]), 1, int(p.L[l]), k, p.seed)
        assert abs(rho[pi, e, 0, l, k] - r_o) <= RHO_TOL
