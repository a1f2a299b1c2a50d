"""Helpers shared by the parity tests: run a problem through the C ABI with the
per-unit outputs, walk its units in output order, and compare with the oracle."""

from __future__ import annotations

import numpy as np

import oracle

RHO_TOL = 1e-4          # |delta rho| bound
XHAT_RTOL = 1e-5        # per-point relative bound on Xhat
XHAT_FLOOR = 1e-3       # denominator floor, as a fraction of std(target)


def units(p):
    """Yield (unit index, j, i, E, tau, L, k, n_m) in the order of rho."""
    u = 0
    for (j, i) in p.pairs:
        for E in p.E:
            for tau in p.tau:
                n_m = p.n - (int(E) - 1) * int(tau)
                for L in p.L:
                    for k in range(p.r):
                        yield u, int(j), int(i), int(E), int(tau), int(L), k, n_m
                        u += 1


def run_detailed(ccm, ctx, p, flags=0):
    """rho [grid], libraries, neighbours and predictions (flat, unit order)."""
    plan = ccm.plan_problem(ctx, p, flags)
    try:
        info = ccm.ccm_plan_get_info(plan)
        rho = np.zeros(ccm.rho_shape(p))
        lib = np.zeros(info["library_entries"], np.int32)
        nbr = np.zeros(info["neighbour_entries"], np.int32)
        xh = np.zeros(info["n_queries"], np.float32)
        ccm.ccm_run_ex(plan, p.series, rho, libraries=lib, neighbours=nbr, predictions=xh)
    finally:
        ccm.ccm_plan_destroy(plan)
    return rho, lib, nbr, xh


def split(p, lib, nbr, xh):
    """Per-unit views of the flat debug outputs."""
    lo = no = qo = 0
    for u, j, i, E, tau, L, k, n_m in units(p):
        yield (u, j, i, E, tau, L, k, n_m, lib[lo:lo + L],
               nbr[no:no + n_m * (E + 1)].reshape(n_m, E + 1), xh[qo:qo + n_m])
        lo += L
        no += n_m * (E + 1)
        qo += n_m


def xhat_rel_err(got, want, target):
    den = np.maximum(np.abs(want), XHAT_FLOOR * np.std(target.astype(np.float64)))
    return float(np.max(np.abs(got.astype(np.float64) - want) / den)) if len(want) else 0.0


def check_units(p, rho, lib, nbr, xh, which=None):
    """Compare every (or the selected) unit with the oracle; returns max errors."""
    flat = rho.reshape(-1)
    worst_rho = worst_x = 0.0
    for (u, j, i, E, tau, L, k, n_m, l_g, n_g, x_g) in split(p, lib, nbr, xh):
        if which is not None and u not in which:
            continue
        r_o, l_o, n_o, x_o = oracle.ccm_unit(p.series, j, i, E, tau, L, k, p.seed, keep=True,
                                             theiler=getattr(p, "theiler", 0),
                                             weight_floor=getattr(p, "weight_floor", 0.0))
        assert np.array_equal(l_g, l_o), f"library differs in unit {u}"
        assert np.array_equal(n_g, n_o), f"neighbours differ in unit {u} " \
            f"(first row {np.nonzero(np.any(n_g != n_o, axis=1))[0][:3]})"
        ex = xhat_rel_err(x_g, x_o, p.series[i])
        assert ex <= XHAT_RTOL, f"Xhat error {ex} in unit {u}"
        if np.isnan(r_o):
            assert np.isnan(flat[u])
        else:
            assert abs(flat[u] - r_o) <= RHO_TOL, f"rho {flat[u]} vs {r_o} in unit {u}"
            worst_rho = max(worst_rho, abs(flat[u] - r_o))
        worst_x = max(worst_x, ex)
    return worst_rho, worst_x
