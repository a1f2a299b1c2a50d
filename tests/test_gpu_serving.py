"""Serving path (ccm_submit / ccm_poll) on the GPU: continuous batching of jobs
of different lengths, E, tau and L grids; admission by device footprint.

The central check: every job's rho is the same whether it runs alone (ccm_run
of its own plan) or inside a batch with other jobs while further jobs arrive.
"""

from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
from paper_1905_00565_gb300 import inputs as I
from tests.ccm_check import RHO_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ccm():
    from paper_1905_00565_gb300 import ccm as c
    return c


def small_jobs(n_jobs=12, seed=7):
    """A served stream scaled down (lengths 500..3000) so that every job is quick."""
    return I.job_stream(n_jobs=n_jobs, rate_per_s=50.0, seed=seed, min_len=500, max_len=3000)


def run_alone(ccm, ctx, p):
    plan = ccm.plan_problem(ctx, p)
    try:
        rho = np.zeros(ccm.rho_shape(p))
        ccm.ccm_run(plan, p.series, rho)
    finally:
        ccm.ccm_plan_destroy(plan)
    return rho


def wait(ccm, ctx, ticket, shape, timeout_s=120):
    rho = np.zeros(shape)
    t0 = time.time()
    while True:
        st = ccm.ccm_poll(ctx, ticket, rho, 200)
        if st == ccm.CCM_OK:
            return rho
        assert time.time() - t0 < timeout_s, "job did not finish"


def wait_times(ccm, ctx, ticket, timeout_s=120):
    """Block until the job has finished; (submit, start, finish) on the context clock."""
    t0 = time.time()
    while True:
        st, sub, start, fin = ccm.ccm_job_times(ctx, ticket)
        if st == ccm.CCM_OK:
            return sub, start, fin
        assert time.time() - t0 < timeout_s, "job did not finish"
        time.sleep(0.002)


def test_each_job_same_alone_and_in_the_mix(ccm):
    """A long job runs; small jobs of other lengths/E/tau/L grids arrive meanwhile,
    are admitted while it is still on the GPU, and every result equals the
    job's result when run alone."""
    long_job = I.subproblem(I.sweep_problem(), E=[9], tau=[0], L=[18, 19], r=250)
    jobs = small_jobs()
    ctx = ccm.ccm_context_create(0)
    try:
        ref_long = run_alone(ccm, ctx, long_job)
        alone = [run_alone(ccm, ctx, j.problem) for j in jobs]
        p = long_job
        t_long = ccm.ccm_submit(ctx, p.series, p.pairs, p.E, p.tau, p.L, p.r, p.seed)
        tickets = []
        for j in jobs:
            q = j.problem
            tickets.append(ccm.ccm_submit(ctx, q.series, q.pairs, q.E, q.tau, q.L, q.r, q.seed))
        _, long_start, long_fin = wait_times(ccm, ctx, t_long)
        starts = []
        for t, j, ref in zip(tickets, jobs, alone):
            _, start, fin = wait_times(ccm, ctx, t)
            starts.append(start)
            got = wait(ccm, ctx, t, ccm.rho_shape(j.problem))
            assert np.max(np.abs(got - ref)) <= 1e-12, j.problem.name
        got_long = wait(ccm, ctx, t_long, ccm.rho_shape(long_job))
        assert np.max(np.abs(got_long - ref_long)) <= 1e-12
        # continuous batching: later arrivals were admitted before the long job ended
        assert min(starts) < long_fin
    finally:
        ccm.ccm_context_destroy(ctx)
    # a couple of units against the oracle as well
    p = jobs[0].problem
    for k in range(2):
        r_o = oracle.ccm_unit(p.series, 1, 0, int(p.E[0]), int(p.tau[0]), int(p.L[0]), k, p.seed)
        assert abs(alone[0][0, 0, 0, 0, k] - r_o) <= RHO_TOL


def test_admission_by_footprint_and_refusals(ccm):
    jobs = small_jobs(8, seed=11)
    # a budget that holds about two jobs at a time: the rest wait, none fails
    big = max(jobs, key=lambda j: j.problem.n_units() * j.problem.n)
    probe_ctx = ccm.ccm_context_create(0)
    plan = ccm.plan_problem(probe_ctx, big.problem)
    foot = ccm.ccm_plan_get_info(plan)["device_bytes"]
    ccm.ccm_plan_destroy(plan)
    ccm.ccm_context_destroy(probe_ctx)
    ctx = ccm.ccm_context_create(0, int(2.5 * foot))
    try:
        tickets = []
        for j in jobs:
            p = j.problem
            tickets.append(ccm.ccm_submit(ctx, p.series, p.pairs, p.E, p.tau, p.L, p.r, p.seed))
        for t, j in zip(tickets, jobs):
            wait(ccm, ctx, t, ccm.rho_shape(j.problem))
        # a job larger than the whole budget is refused at submit
        huge = I.sweep_problem()
        with pytest.raises(ccm.CCMError) as ei:
            ccm.ccm_submit(ctx, huge.series, huge.pairs, huge.E, huge.tau, huge.L, huge.r,
                           huge.seed)
        assert ei.value.status == ccm.CCM_ETOOLARGE
        with pytest.raises(ccm.CCMError) as ei:
            ccm.ccm_poll(ctx, 987654321, np.zeros(1), 0)
        assert ei.value.status == ccm.CCM_ENOTFOUND
    finally:
        ccm.ccm_context_destroy(ctx)


def test_cancel_a_queued_job(ccm):
    p = I.subproblem(I.sweep_problem(), E=[9], tau=[0], L=[19], r=60)
    probe_ctx = ccm.ccm_context_create(0)
    plan = ccm.plan_problem(probe_ctx, p)
    foot = ccm.ccm_plan_get_info(plan)["device_bytes"]
    ccm.ccm_plan_destroy(plan)
    ccm.ccm_context_destroy(probe_ctx)
    ctx = ccm.ccm_context_create(0, int(1.5 * foot))    # one long job at a time
    try:
        first = [ccm.ccm_submit(ctx, p.series, p.pairs, p.E, p.tau, p.L, p.r, p.seed)
                 for _ in range(3)]
        q = I.Problem(series=I.logistic_pair(300), pairs=I.BOTH_DIRECTIONS.copy(),
                      E=np.array([2], np.int32), tau=np.array([1], np.int32),
                      L=np.array([20], np.int64), r=2, seed=3, name="tiny")
        t = ccm.ccm_submit(ctx, q.series, q.pairs, q.E, q.tau, q.L, q.r, q.seed)
        assert ccm.ccm_cancel(ctx, t) == ccm.CCM_OK       # still queued behind the long jobs
        with pytest.raises(ccm.CCMError) as ei:
            ccm.ccm_poll(ctx, t, np.zeros(ccm.rho_shape(q)), 60_000)
        assert ei.value.status == ccm.CCM_ECANCELLED
        for f in first:
            wait(ccm, ctx, f, ccm.rho_shape(p))
    finally:
        ccm.ccm_context_destroy(ctx)


def test_a_failed_batch_fails_only_its_own_jobs(ccm, monkeypatch):
    """Host-side fault injection (no device fault): the context's second batch
    fails its launch as if a CUDA call had returned an error.  Its job reports
    CCM_ECUDA at ccm_poll; the jobs before and after it, and later batches on
    the same context, finish with the rho they have when run alone."""
    jobs = small_jobs(4, seed=13)
    monkeypatch.setenv("CCM_FAULT_INJECT_BATCH", "1")
    ctx = ccm.ccm_context_create(0)
    monkeypatch.delenv("CCM_FAULT_INJECT_BATCH")
    try:
        alone = [run_alone(ccm, ctx, j.problem) for j in jobs]
        results = []
        for n, (j, ref) in enumerate(zip(jobs, alone)):
            q = j.problem
            t = ccm.ccm_submit(ctx, q.series, q.pairs, q.E, q.tau, q.L, q.r, q.seed)
            wait_times(ccm, ctx, t)               # one job per batch: batch n is job n
            rho = np.zeros(ccm.rho_shape(q))
            if n == 1:
                with pytest.raises(ccm.CCMError) as ei:
                    ccm.ccm_poll(ctx, t, rho, 0)
                assert ei.value.status == ccm.CCM_ECUDA
                assert "injected" in str(ei.value)
            else:
                assert ccm.ccm_poll(ctx, t, rho, 0) == ccm.CCM_OK
                assert np.array_equal(rho, ref), q.name
                results.append(n)
        assert results == [0, 2, 3]
        # the failed batch released its share of the budget: a big job still fits
        p = I.subproblem(I.sweep_problem(), E=[3], tau=[0], L=[5], r=20)
        t = ccm.ccm_submit(ctx, p.series, p.pairs, p.E, p.tau, p.L, p.r, p.seed)
        assert np.array_equal(wait(ccm, ctx, t, ccm.rho_shape(p)), run_alone(ccm, ctx, p))
    finally:
        ccm.ccm_context_destroy(ctx)
