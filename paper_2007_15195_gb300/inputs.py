"""Seeded synthetic inputs for the Vecchia log-CDF workloads.

This module holds no arithmetic of the method (no ordering, no neighbour
search, no covariance, no CDF): it draws raw sites, thresholds and covariance
parameters with numpy's Philox bit generator, one stream per array, so that
the CUDA path and the oracle read the same inputs.  The workloads follow the
spatial settings of the paper's simulation study (Sec. 3: sites on regular
grids in the unit square, exponential covariance with unit variance) widened
to the sizes this library is measured at.
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

# Stream identifiers: each array of a workload draws from its own stream.
_STREAM_SITES, _STREAM_U, _STREAM_D, _STREAM_RANGE, _STREAM_M, _STREAM_NU, _STREAM_ARRIVAL = range(7)

# Phi^{-1}(0.9), the standard normal 0.9 quantile (a textbook constant).
Z_090 = 1.2815515655446004

COV_EXPONENTIAL, COV_MATERN = 0, 1


def rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence([int(seed), int(stream)])))


@dataclass
class Problem:
    """One log-CDF problem: raw (unordered) sites, centred thresholds, covariance."""
    sites: np.ndarray            # D x 2 float64
    u: np.ndarray                # D float64, per raw site
    cov: tuple                   # (kind, variance, range, nu, nugget)
    m: int
    N: int
    S: int
    seed: int = 0
    order: str = "xy"            # "xy" | "maxmin" | "identity"
    name: str = ""

    @property
    def D(self) -> int:
        return int(self.sites.shape[0])


def grid_sites(n: int) -> np.ndarray:
    """n x n regular grid on [0,1]^2, x then y ascending: coordinates k/(n-1)."""
    t = np.arange(n, dtype=np.float64) / (n - 1)
    xx, yy = np.meshgrid(t, t, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel()], axis=1)


def uniform_sites(D: int, seed: int, stream_offset: int = 0) -> np.ndarray:
    return rng(seed, _STREAM_SITES + 16 * stream_offset).random((D, 2))


def grid10(seed: int = 0) -> Problem:
    """10x10 grid, exponential range 0.2, unit variance, orthant u = 0, m = 10,
    N = 2,000 lattice points x S = 10 shifts."""
    s = grid_sites(10)
    return Problem(s, np.zeros(100), (COV_EXPONENTIAL, 1.0, 0.2, 0.5, 0.0), m=10, N=2000, S=10,
                   seed=seed, order="xy", name="grid10_exp0.2_m10")


def grid50(m: int = 20, seed: int = 0, workload_seed: int = 0, N: int = 4096, S: int = 16) -> Problem:
    """50x50 grid, Matern nu=1.5 range 0.1, unit variance, u_i ~ N(0.5, 0.25^2),
    N = 4,096 x S = 16."""
    s = grid_sites(50)
    u = rng(workload_seed, _STREAM_U).normal(0.5, 0.25, size=2500)
    return Problem(s, u, (COV_MATERN, 1.0, 0.1, 1.5, 0.0), m=m, N=N, S=S, seed=seed, order="xy",
                   name="grid50_matern1.5_m%d" % m)


def grid100(seed: int = 0, workload_seed: int = 0, N: int = 2048, S: int = 8) -> Problem:
    """100x100 grid (the joint-group experiment's grid, Sec. 3.2), exponential
    range 0.1 with unit variance, u_i ~ N(0.5, 0.25^2), N = 2,048 x S = 8.
    m is set by the caller (per group member)."""
    s = grid_sites(100)
    u = rng(workload_seed, _STREAM_U).normal(0.5, 0.25, size=10000)
    return Problem(s, u, (COV_EXPONENTIAL, 1.0, 0.1, 0.5, 0.0), m=0, N=N, S=S, seed=seed, order="xy",
                   name="grid100_exp0.1")


@dataclass
class CensoredReplicate:
    """One replicate of a censored likelihood: values at the sites, the ones
    above the threshold observed (x_obs at sites_obs), the others censored at
    the threshold (x_cen = threshold at sites_cen)."""
    sites_cen: np.ndarray
    x_cen: np.ndarray
    sites_obs: np.ndarray
    x_obs: np.ndarray


def censored_replicates(n_rep: int = 32, D: int = 528, frac_obs: float = 0.1, workload_seed: int = 0):
    """The application's shape (Sec. 4.1): D = 528 station sites uniform in the
    unit square (a stand-in for the stations, which are not available), the
    anisotropic exponential covariance of Sec. 4.1 (range 0.2, angle 0.5,
    aspect 1.5, unit variance), and per replicate a random frac_obs of the
    sites above the threshold Phi^{-1}(0.9): their values are the threshold
    plus Exp(1)/2, the others are censored at the threshold.  Returns the
    covariance tuple and the replicates (sites not ordered)."""
    s = rng(workload_seed, _STREAM_SITES).random((D, 2))
    g = rng(workload_seed, _STREAM_M)
    e = rng(workload_seed, _STREAM_U)
    cov = (2, 1.0, 0.2, 0.5, 0.0, 0.5, 1.5)  # VECCHIA_COV_ANISO_EXP
    reps = []
    for _ in range(n_rep):
        k = max(1, int(round(frac_obs * D)))
        obs = np.sort(g.choice(D, size=k, replace=False))
        cen = np.setdiff1d(np.arange(D), obs)
        reps.append(CensoredReplicate(s[cen].copy(), np.full(cen.size, Z_090), s[obs].copy(),
                                      Z_090 + 0.5 * e.exponential(size=k)))
    return cov, reps


def batch_problems(n_problems: int = 4096, workload_seed: int = 0, m: int = 20, N: int = 2048,
                   S: int = 8, d_lo: float = 50.0, d_hi: float = 2000.0) -> List[Problem]:
    """Independent problems: D log-uniform in [d_lo, d_hi], sites uniform in the
    unit square, exponential covariance with range ~ U[0.05, 0.5], u_i = Phi^{-1}(0.9)."""
    Ds = np.rint(np.exp(rng(workload_seed, _STREAM_D).uniform(np.log(d_lo), np.log(d_hi),
                                                              size=n_problems))).astype(np.int64)
    ranges = rng(workload_seed, _STREAM_RANGE).uniform(0.05, 0.5, size=n_problems)
    out = []
    for p in range(n_problems):
        s = uniform_sites(int(Ds[p]), workload_seed, stream_offset=p + 1)
        out.append(Problem(s, np.full(int(Ds[p]), Z_090), (COV_EXPONENTIAL, 1.0, float(ranges[p]), 0.5, 0.0),
                           m=m, N=N, S=S, seed=p, order="maxmin", name="batch%d" % p))
    return out


def large(D: int = 100_000, nu: float = 1.5, workload_seed: int = 0, m: int = 30, N: int = 8192,
          S: int = 16) -> Problem:
    """D uniform sites, Matern nu in {0.5, 1.5} range 0.05, u_i ~ U[0, 2], maxmin order."""
    s = uniform_sites(D, workload_seed)
    u = rng(workload_seed, _STREAM_U).uniform(0.0, 2.0, size=D)
    return Problem(s, u, (COV_MATERN, 1.0, 0.05, float(nu), 0.0), m=m, N=N, S=S, seed=0,
                   order="maxmin", name="large%d_matern%g" % (D, nu))


@dataclass
class Request:
    arrival_s: float
    problem: Problem


def serving_stream(n_requests: int = 20_000, rate_hz: float = 2000.0, workload_seed: int = 0,
                   d_lo: float = 100.0, d_hi: float = 50_000.0, N: int = 2048, S: int = 8,
                   max_D: Optional[int] = None) -> List[Request]:
    """Poisson arrivals; D log-uniform in [d_lo, d_hi]; m in {10, 20, 30};
    covariance parameters along a synthetic optimiser trajectory: the range does
    a seeded random walk clipped to [0.05, 0.5], nu alternates in blocks between
    0.5 and 1.5.  Sites uniform in the unit square; u_i = Phi^{-1}(0.9)."""
    r_arr = rng(workload_seed, _STREAM_ARRIVAL)
    gaps = r_arr.exponential(1.0 / rate_hz, size=n_requests)
    t = np.cumsum(gaps)
    Ds = np.rint(np.exp(rng(workload_seed, _STREAM_D).uniform(np.log(d_lo), np.log(d_hi),
                                                              size=n_requests))).astype(np.int64)
    if max_D is not None:
        Ds = np.minimum(Ds, max_D)
    ms = rng(workload_seed, _STREAM_M).choice(np.array([10, 20, 30]), size=n_requests)
    steps = rng(workload_seed, _STREAM_RANGE).normal(0.0, 0.02, size=n_requests)
    nus = rng(workload_seed, _STREAM_NU).integers(0, 2, size=(n_requests + 63) // 64)
    rho = 0.2
    out = []
    for k in range(n_requests):
        rho = float(np.clip(rho + steps[k], 0.05, 0.5))
        nu = 0.5 if nus[k // 64] == 0 else 1.5
        s = uniform_sites(int(Ds[k]), workload_seed, stream_offset=k + 1)
        out.append(Request(float(t[k]), Problem(s, np.full(int(Ds[k]), Z_090), (COV_MATERN, 1.0, rho, nu, 0.0),
                                                m=int(ms[k]), N=N, S=S, seed=k, order="maxmin",
                                                name="req%d" % k)))
    return out


def small_random(D: int, seed: int, m: int, cov=(COV_EXPONENTIAL, 1.0, 0.3, 0.5, 0.0), u_mean: float = 0.3,
                 u_sd: float = 0.5, N: int = 512, S: int = 4, order: str = "maxmin") -> Problem:
    """Small random problem for parity tests (sites uniform, u ~ N(u_mean, u_sd^2))."""
    s = uniform_sites(D, seed)
    u = rng(seed, _STREAM_U).normal(u_mean, u_sd, size=D)
    return Problem(s, u, cov, m=m, N=N, S=S, seed=seed, order=order, name="small%d_%d" % (D, seed))
