"""Long weakly coupled series (N = 10^5, library tiled through shared memory):
parity at full size on sampled outputs (needs a GB300).

The oracle cannot afford all 10^5 queries against L = 50000 in seconds, so per
realization it recomputes a seeded sample of query points one by one
(neighbours bit-exact against its FP32 selection; against its FP64 selection
identical except at near ties below 1e-6 relative; predictions within 1e-5).
Over all N_m queries it replays the GPU's neighbour sets (simplex prediction in
FP64 from the given sets, then the skill), which checks every prediction and
rho; rho is also checked against the plain comparator (same neighbours, one CTA
two-pass Pearson).
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1905_00565_gb300 import inputs as I
from tests.ccm_check import NEAR_TIE, RHO_TOL, XHAT_RTOL, run_detailed, split, xhat_rel_err

pytestmark = pytest.mark.gpu


def test_long_series_sampled_parity():
    from paper_1905_00565_gb300 import ccm
    base = I.long_series_problem()
    p = I.Problem(series=base.series, pairs=base.pairs, E=np.array([3, 6], np.int32),
                  tau=np.array([1], np.int32), L=np.array([1000, 50000], np.int64), r=1,
                  seed=base.seed, name="long-sample")
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
    rng = np.random.default_rng(2)
    flat = rho.reshape(-1)
    for (u, j, i, E, tau, L, k, n_m, l_g, n_g, x_g) in split(p, lib, nbr, xh):
        assert np.array_equal(l_g, oracle.library(n_m, L, j, E, tau, k, p.seed))
        q = np.sort(rng.choice(n_m, size=300, replace=False))
        q = np.concatenate([[0, n_m - 1], q])
        nb_o, xh_o = oracle.query_subset(p.series[j], p.series[i], E, tau, l_g, q)
        assert np.array_equal(n_g[q], nb_o), f"neighbours differ in unit {u}"
        assert xhat_rel_err(x_g[q], xh_o, p.series[i]) <= XHAT_RTOL
        # FP64 selection: other sets only at near ties
        nb_64, _ = oracle.query_subset(p.series[j], p.series[i], E, tau, l_g, q,
                                       select_fp64=True)
        differ = q[np.any(np.sort(n_g[q], 1) != np.sort(nb_64, 1), axis=1)]
        if len(differ):
            assert np.all(oracle.query_margin(p.series[j], E, tau, l_g, differ) < NEAR_TIE)
        # every query: the oracle's prediction and skill from the GPU's sets
        x_rep = oracle.predict(p.series[j], p.series[i], E, tau, n_g)
        assert xhat_rel_err(x_g, x_rep, p.series[i]) <= XHAT_RTOL
        assert abs(flat[u] - oracle.skill(p.series[i], E, tau, x_rep)) <= RHO_TOL
        assert abs(flat[u] - rho_plain.reshape(-1)[u]) <= 1e-12
    assert np.all(np.isfinite(rho))
