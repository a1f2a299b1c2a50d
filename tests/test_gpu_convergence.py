"""Convergence decision on the GPU (ccm_convergence) against the oracle, bit
for bit: random grids with NaN, ties and an unsorted L axis, a real CCM
sweep's rho left on the device, device output, and the argument checks
(needs a GB300)."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1905_00565_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccm():
    from paper_1905_00565_gb300 import ccm as c
    return c


def as_rows(res):
    return np.stack([res[f].astype(np.float64) for f in
                     ("rho_first", "rho_last", "jt", "z", "n_valid", "converged")], axis=-1)


def same(got, want):
    """Bit-equal, NaN equal to NaN."""
    return np.array_equal(got, want, equal_nan=True)


def test_random_grids_match_oracle_bit_for_bit(ccm):
    rng = np.random.default_rng(21)
    ctx = ccm.ccm_context_create(0)
    try:
        for n_L, r in [(2, 1), (3, 7), (20, 250), (64, 384), (5, 4000)]:
            rho = rng.normal(0.3, 0.2, size=(3, 2, n_L, r))
            rho += np.linspace(0, 0.2, n_L)[:, None] * rng.random()     # some trend
            rho[rng.random(rho.shape) < 0.02] = np.nan
            rho[..., 0, :3] = 0.25                                      # ties
            rho[..., -1, :3] = 0.25
            L = rng.permutation(np.arange(10, 10 + 37 * n_L, 37))
            got = as_rows(ccm.ccm_convergence(ctx, rho, L))
            assert same(got, oracle.convergence(rho, L)), (n_L, r)
    finally:
        ccm.ccm_context_destroy(ctx)


def test_sweep_rho_on_device(ccm):
    torch = pytest.importorskip("torch")
    base = I.sweep_problem()
    p = I.subproblem(base, E=[1, 4], tau=[0, 2], r=40)
    ctx = ccm.ccm_context_create(0)
    try:
        plan = ccm.plan_problem(ctx, p, ccm.CCM_INPUT_ON_DEVICE | ccm.CCM_OUTPUT_ON_DEVICE)
        try:
            s = torch.from_numpy(p.series).cuda()
            rho = torch.zeros(ccm.rho_shape(p), dtype=torch.float64, device="cuda")
            ccm.ccm_run(plan, s, rho)
            torch.cuda.synchronize()
        finally:
            ccm.ccm_plan_destroy(plan)
        got = as_rows(ccm.ccm_convergence(ctx, rho, p.L))
        out = torch.zeros(got[..., 0].size * 40, dtype=torch.uint8, device="cuda")
        ccm.ccm_convergence(ctx, rho, p.L, out=out)
        torch.cuda.synchronize()
        dev = np.frombuffer(out.cpu().numpy().tobytes(), dtype=ccm._CONV_DTYPE)
        assert same(as_rows(dev).reshape(got.shape), got)
    finally:
        ccm.ccm_context_destroy(ctx)
    want = oracle.convergence(rho.cpu().numpy(), p.L)
    assert same(got, want)
    # the coupled logistic map: cross-mapping x from M_y (y is driven by x)
    # converges at every (E, tau) of the subset
    assert np.all(got[0, ..., 5] == 1.0)


def test_arguments_are_checked(ccm):
    ctx = ccm.ccm_context_create(0)
    try:
        for rho, L in [(np.zeros((2, 1, 5)), [10]),                  # n_L = 1
                       (np.zeros((2, 65, 2)), np.arange(65) + 5),    # n_L > 64
                       (np.zeros((1, 10, 2500)), np.arange(10) + 5),  # n_L * r > 24576
                       (np.zeros((1, 3, 4)), [5, 9, 5])]:              # repeated L
            with pytest.raises(ccm.CCMError) as ei:
                ccm.ccm_convergence(ctx, rho, L)
            assert ei.value.status == ccm.CCM_EINVAL
    finally:
        ccm.ccm_context_destroy(ctx)
