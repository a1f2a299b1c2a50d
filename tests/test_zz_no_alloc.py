"""ccm_run_noalloc: one CCM cell with no device allocation (needs a GB300).

Callers that cannot call cudaMalloc at run time -- a framework whose caching
allocator already owns the device memory, or a latency-critical loop that must
not let cudaMalloc/cudaFree synchronise the device -- use this entry point;
it keeps all scratch in the library's fixed device array.  These checks call
it through the C ABI twice in a row per cell and compare with ccm_run, the
planned entry point, within the rho tolerance of the other parity tests.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""

from __future__ import annotations

import numpy as np
import pytest

from paper_1905_00565_gb300 import inputs as I
from tests.ccm_check import RHO_TOL

pytestmark = pytest.mark.gpu


def test_noalloc_matches_ccm_run_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    from paper_1905_00565_gb300 import ccm
    p = I.sweep_problem()                       # N = 10^4
    cells = [(1, 0, 3, 2, 2000, 8),             # (j, i, E, tau, L, r)
             (0, 1, 10, 1, 9000, 4),            # several library tiles
             (1, 0, 1, 4, 100, 16)]
    ctx = ccm.ccm_context_create(0)
    try:
        s_dev = torch.from_numpy(p.series).cuda()
        for (j, i, E, tau, L, r) in cells:
            plan = ccm.ccm_plan(ctx, p.series.shape, [[j, i]], [E], [tau], [L], r, p.seed)
            want = np.zeros((1, 1, 1, 1, r))
            try:
                ccm.ccm_run(plan, p.series, want)
            finally:
                ccm.ccm_plan_destroy(plan)
            want = want.reshape(-1)
            for _ in range(2):
                rho = torch.full((r,), float("nan"), dtype=torch.float64, device="cuda")
                ccm.ccm_run_noalloc(s_dev, j, i, E, tau, L, r, p.seed, rho)
                got = rho.cpu().numpy()
                assert np.all(np.isfinite(got))
                assert np.max(np.abs(got - want)) <= RHO_TOL, (j, i, E, tau, L, r)
    finally:
        ccm.ccm_context_destroy(ctx)


def test_noalloc_long_manifold_matches_ccm_run():
    """N = 10^5: a manifold above the one-pass sort size keeps time order here (no
    scratch for the merge sort) while ccm_run sorts it, and the sampler recomputes
    its keys per radix pass (more points than fit in shared memory); about 1.3 MB
    of the fixed scratch.  Two calls in a row, each against ccm_run."""
    torch = pytest.importorskip("torch")
    from paper_1905_00565_gb300 import ccm
    p = I.long_series_problem()
    j, i, E, tau, L, r = 1, 0, 4, 1, 1000, 4
    ctx = ccm.ccm_context_create(0)
    try:
        plan = ccm.ccm_plan(ctx, p.series.shape, [[j, i]], [E], [tau], [L], r, p.seed)
        want = np.zeros((1, 1, 1, 1, r))
        try:
            ccm.ccm_run(plan, p.series, want)
        finally:
            ccm.ccm_plan_destroy(plan)
    finally:
        ccm.ccm_context_destroy(ctx)
    want = want.reshape(-1)
    s_dev = torch.from_numpy(p.series).cuda()
    for _ in range(2):
        rho = torch.full((r,), float("nan"), dtype=torch.float64, device="cuda")
        ccm.ccm_run_noalloc(s_dev, j, i, E, tau, L, r, p.seed, rho)
        got = rho.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - want)) <= RHO_TOL


def test_noalloc_rejects_a_cell_beyond_its_fixed_scratch():
    torch = pytest.importorskip("torch")
    from paper_1905_00565_gb300 import ccm
    s_dev = torch.zeros((2, 100_000), dtype=torch.float32, device="cuda")
    rho = torch.zeros(250, dtype=torch.float64, device="cuda")
    with pytest.raises(ccm.CCMError) as ei:       # 250 libraries of 50000 points: 50 MB
        ccm.ccm_run_noalloc(s_dev, 1, 0, 3, 1, 50_000, 250, 1, rho)
    assert ei.value.status == ccm.CCM_ETOOLARGE
    assert "scratch" in str(ei.value)
    with pytest.raises(ccm.CCMError) as ei:
        ccm.ccm_run_noalloc(s_dev, 1, 1, 3, 1, 100, 4, 1, rho)
    assert ei.value.status == ccm.CCM_EINVAL
