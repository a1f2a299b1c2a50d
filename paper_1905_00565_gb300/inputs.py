"""Seeded synthetic inputs for CCM: coupled logistic maps and CCM problem grids.

This module holds no CCM arithmetic.  It makes the series that CCM is run on
and the parameter grids (E, tau, L, r) of the five standard workloads, so that
the CUDA path, the CPU oracle, the tests and the benchmark all consume the
same FP32 arrays.  Every series is iterated in FP64 on the host and stored as
FP32; the trajectories only need to be reproducible here, not to match any
other program.

The paper (Sect. 4) runs CCM on one unnamed series of length 4000 with r=500,
L in {500,1000,2000} and E, tau in {1,2,4}; that data is not available, so the
two-species coupled logistic map of the method's source (Sugihara et al. 2012,
cited in Sect. 2.1) and the networks below stand in for it.

Variable / pair convention: a *pair* is ``(j, i)`` = (library variable whose
shadow manifold is searched, target variable that is cross-mapped).  For two
series stored as rows ``[X, Y]``, pair ``(1, 0)`` builds the library from M_Y
and predicts X, which tests "X drives Y" (Sect. 2.1: information on a driver
is encoded in the driven variable's reconstructed state space).
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

DEFAULT_SEED = 20190501


@dataclasses.dataclass
class Problem:
    """A CCM sweep: series [V][N] FP32 plus the (pair, E, tau, L, r) grid."""

    series: np.ndarray           # float32 [V][N], C-contiguous
    pairs: np.ndarray            # int32 [n_pairs][2] = (library var j, target var i)
    E: np.ndarray                # int32 [n_E], each in 1..10
    tau: np.ndarray              # int32 [n_tau], each >= 1
    L: np.ndarray                # int64 [n_L]
    r: int                       # realizations per (pair, E, tau, L) cell
    seed: int                    # library sampler seed
    name: str = ""
    theiler: int = 0             # exclusion window W (0: only the query itself)
    weight_floor: float = 0.0    # simplex weight floor f (0: none)

    @property
    def n_series(self) -> int:
        return int(self.series.shape[0])

    @property
    def n(self) -> int:
        return int(self.series.shape[1])

    def n_units(self) -> int:
        return len(self.pairs) * len(self.E) * len(self.tau) * len(self.L) * self.r

    def unit_grid(self):
        """Yield (p, e, t, l) index tuples in the output order of rho."""
        for p in range(len(self.pairs)):
            for e in range(len(self.E)):
                for t in range(len(self.tau)):
                    for l in range(len(self.L)):
                        yield p, e, t, l

    def queries(self) -> int:
        """Neighbour queries in the whole sweep (all manifold points of every unit)."""
        tot = 0
        for _, e, t, _ in self.unit_grid():
            tot += self.n - (int(self.E[e]) - 1) * int(self.tau[t])
        return tot * self.r

    def pair_count(self) -> int:
        """Query-library point pairs of a brute-force sweep (sum over units of N_m * L)."""
        tot = 0
        for _, e, t, l in self.unit_grid():
            tot += (self.n - (int(self.E[e]) - 1) * int(self.tau[t])) * int(self.L[l])
        return tot * self.r

    def flop_count(self) -> int:
        """Algorithmic FP32 flops of the distance step: 3E per query-library pair."""
        tot = 0
        for _, e, t, l in self.unit_grid():
            Ev = int(self.E[e])
            tot += (self.n - (Ev - 1) * int(self.tau[t])) * int(self.L[l]) * 3 * Ev
        return tot * self.r


def logistic_pair(n: int, rx: float = 3.8, ry: float = 3.5, bxy: float = 0.02,
                  byx: float = 0.1, x0: float = 0.4, y0: float = 0.2) -> np.ndarray:
    """Two-species coupled logistic map, rows [X, Y], float32 [2][n].

    X(t+1) = X(t) (rx - rx X(t) - bxy Y(t)),  Y(t+1) = Y(t) (ry - ry Y(t) - byx X(t)),
    X(0)=x0, Y(0)=y0, iterated in FP64 and stored in FP32.
    """
    out = np.empty((2, n), dtype=np.float64)
    x, y = float(x0), float(y0)
    for t in range(n):
        out[0, t] = x
        out[1, t] = y
        x, y = x * (rx - rx * x - bxy * y), y * (ry - ry * y - byx * x)
    if not np.all(np.isfinite(out)):
        raise ValueError("logistic map diverged; choose other parameters")
    return np.ascontiguousarray(out.astype(np.float32))


def logistic_network(V: int = 64, n: int = 5000, density: float = 0.05,
                     seed: int = DEFAULT_SEED + 5, max_tries: int = 1000
                     ) -> Tuple[np.ndarray, int]:
    """64-variable coupled logistic network, float32 [V][n], and the accepted seed.

    x_i(t+1) = x_i(t) (r_i - r_i x_i(t) - sum_j beta_ij x_j(t)) with r_i ~ U(3.6, 3.9),
    beta_ii = 0, each off-diagonal beta_ij present with probability ``density`` and
    then ~ U(0, 0.1), x_i(0) ~ U(0.1, 0.9).  Some draws leave (0, 1) and run off to
    -inf; such a draw is rejected and redrawn with seed+1, seed+2, ... until every
    trajectory stays in (0, 1).  The seed that was accepted is returned.
    """
    for s in range(seed, seed + max_tries):
        rng = np.random.Generator(np.random.Philox(s))
        r = rng.uniform(3.6, 3.9, size=V)
        mask = rng.random((V, V)) < density
        np.fill_diagonal(mask, False)
        beta = np.where(mask, rng.uniform(0.0, 0.1, size=(V, V)), 0.0)
        x = rng.uniform(0.1, 0.9, size=V)
        out = np.empty((V, n), dtype=np.float64)
        ok = True
        for t in range(n):
            out[:, t] = x
            x = x * (r - r * x - beta @ x)
            if not (np.all(np.isfinite(x)) and np.all(x > 0.0) and np.all(x < 1.0)):
                ok = False
                break
        if ok:
            return np.ascontiguousarray(out.astype(np.float32)), s
    raise RuntimeError("no bounded network found")


def add_noise(series: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Add i.i.d. N(0, sigma^2) observation noise (FP64 draw, FP32 result)."""
    rng = np.random.Generator(np.random.Philox(seed))
    noisy = series.astype(np.float64) + rng.normal(0.0, sigma, size=series.shape)
    return np.ascontiguousarray(noisy.astype(np.float32))


def log_grid(lo: float, hi: float, count: int) -> np.ndarray:
    """round(logspace(lo, hi, count)) as int64."""
    return np.round(np.logspace(math.log10(lo), math.log10(hi), count)).astype(np.int64)


BOTH_DIRECTIONS = np.array([[1, 0], [0, 1]], dtype=np.int32)


def plain_ccm_problem(seed: int = DEFAULT_SEED + 1) -> Problem:
    """Plain single-job CCM: N=1000, E=2, tau=1, L in {50,...,800}, r=100, both directions."""
    return Problem(series=logistic_pair(1000), pairs=BOTH_DIRECTIONS.copy(),
                   E=np.array([2], np.int32), tau=np.array([1], np.int32),
                   L=np.array([50, 100, 200, 400, 800], np.int64), r=100, seed=seed,
                   name="plain-ccm-n1000")


def paper_scenario_problem(seed: int = DEFAULT_SEED + 6) -> Problem:
    """The paper's baseline scenario (Sect. 4) on a synthetic stand-in: N=4000,
    r=500, L in {500, 1000, 2000}, E and tau in {1, 2, 4}, both directions of the
    coupled logistic map (the paper's series is unnamed and not available)."""
    return Problem(series=logistic_pair(4000), pairs=BOTH_DIRECTIONS.copy(),
                   E=np.array([1, 2, 4], np.int32), tau=np.array([1, 2, 4], np.int32),
                   L=np.array([500, 1000, 2000], np.int64), r=500, seed=seed,
                   name="paper-baseline-n4000")


def sweep_problem(seed: int = DEFAULT_SEED + 2, n: int = 10_000, r: int = 250) -> Problem:
    """Batched sweep: N=10^4, E=1..10, tau=1..4, 20 L log-spaced 100..9000, r=250."""
    return Problem(series=logistic_pair(n), pairs=BOTH_DIRECTIONS.copy(),
                   E=np.arange(1, 11, dtype=np.int32), tau=np.arange(1, 5, dtype=np.int32),
                   L=log_grid(100, 9000, 20), r=r, seed=seed, name="sweep-n10000")


def long_series_problem(seed: int = DEFAULT_SEED + 3, n: int = 100_000, r: int = 250) -> Problem:
    """Long weakly coupled series: N=10^5, byx=0.01, bxy=0, noise 0.01, E=3..6, tau=1."""
    s = add_noise(logistic_pair(n, bxy=0.0, byx=0.01), 0.01, seed)
    return Problem(series=s, pairs=BOTH_DIRECTIONS.copy(),
                   E=np.array([3, 4, 5, 6], np.int32), tau=np.array([1], np.int32),
                   L=np.array([1000, 5000, 10000, 25000, 50000], np.int64), r=r, seed=seed,
                   name="long-n100000")


def network_problem(seed: int = DEFAULT_SEED + 5, n: int = 5000, r: int = 250) -> Problem:
    """Network sweep: 64 variables, all 4032 ordered pairs, E in {2,3,4}, tau=1, 8 L values."""
    series, used = logistic_network(64, n, 0.05, seed)
    pairs = np.array([[j, i] for j in range(64) for i in range(64) if i != j], np.int32)
    return Problem(series=series, pairs=pairs, E=np.array([2, 3, 4], np.int32),
                   tau=np.array([1], np.int32), L=log_grid(100, 4500, 8), r=r, seed=used,
                   name="network-v64-n5000")


def job_L_grid(n_m: int, E: int) -> np.ndarray:
    """10-point L grid of a served job: L_k = max(E+2, floor(0.09 (k+1) N_m)), k=0..9."""
    return np.array([max(E + 2, int(math.floor(0.09 * (k + 1) * n_m))) for k in range(10)],
                    np.int64)


@dataclasses.dataclass
class Job:
    """One served CCM job and its arrival time (seconds from the stream start)."""

    arrival_s: float
    problem: Problem


def job_stream(n_jobs: int = 2000, rate_per_s: float = 1.0, seed: int = DEFAULT_SEED + 4,
               min_len: int = 500, max_len: int = 50_000) -> List[Job]:
    """Served request stream: Poisson arrivals, per-job coupled logistic pair.

    Each job draws bxy, byx ~ U(0, 0.1), length ~ floor(exp U(ln min_len, ln max_len)),
    E ~ U{1..10}, tau ~ U{1..5}, r in {100, 250}, both directions and the 10-point
    L grid of :func:`job_L_grid`.  Initial values are X0=0.4, Y0=0.2.
    """
    rng = np.random.Generator(np.random.Philox(seed))
    jobs: List[Job] = []
    t = 0.0
    for q in range(n_jobs):
        t += float(rng.exponential(1.0 / rate_per_s))
        bxy, byx = rng.uniform(0.0, 0.1, size=2)
        n = int(math.floor(math.exp(rng.uniform(math.log(min_len), math.log(max_len)))))
        E = int(rng.integers(1, 11))
        tau = int(rng.integers(1, 6))
        r = int(rng.choice([100, 250]))
        n_m = n - (E - 1) * tau
        prob = Problem(series=logistic_pair(n, bxy=float(bxy), byx=float(byx)),
                       pairs=BOTH_DIRECTIONS.copy(), E=np.array([E], np.int32),
                       tau=np.array([tau], np.int32), L=job_L_grid(n_m, E), r=r,
                       seed=seed * 1000 + q, name=f"job{q}")
        jobs.append(Job(arrival_s=t, problem=prob))
    return jobs


def subproblem(p: Problem, pairs: Sequence[int] | None = None, E: Sequence[int] | None = None,
               tau: Sequence[int] | None = None, L: Sequence[int] | None = None,
               r: int | None = None) -> Problem:
    """A smaller grid over the same series (index lists select entries of each axis)."""
    pick = lambda arr, idx: arr if idx is None else np.ascontiguousarray(arr[list(idx)])
    return Problem(series=p.series, pairs=pick(p.pairs, pairs), E=pick(p.E, E),
                   tau=pick(p.tau, tau), L=pick(p.L, L), r=p.r if r is None else r,
                   seed=p.seed, name=p.name + "-sub", theiler=p.theiler,
                   weight_floor=p.weight_floor)
