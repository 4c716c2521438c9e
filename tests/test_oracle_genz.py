"""Pins of the oracle's Genz QMC estimate of a Gaussian CDF.

Sec. 2.2 and Sec. 3 evaluate every low-dimensional CDF by Genz's QMC.  The
oracle's estimate is pinned to closed forms (D = 1, independence, the bi- and
trivariate orthant formula, the equicorrelated rho = 1/2 orthant 1/(D+1)), to
a 1-D quadrature of the bivariate CDF at u != 0, and to brute-force Monte
Carlo for D <= 6.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O
from paper_2007_15195_gb300 import inputs


def _within(p, rel_se, ref, k=4.0, floor=1e-12):
    return abs(p - ref) <= k * abs(p) * rel_se + floor


def test_d1_exact():
    for u, v in [(0.0, 1.0), (1.3, 1.0), (-2.0, 4.0), (5.0, 0.25)]:
        p, rse = O.genz_cdf(np.array([[v]]), [u], 128, 4, 0)
        assert p == O.Phi(u / math.sqrt(v))
        assert rse == 0.0


def test_independence_gives_product_exactly():
    var = np.array([1.0, 2.0, 0.5, 3.0, 1.0])
    u = np.array([0.3, -0.4, 1.1, 0.0, 2.0])
    p, rse = O.genz_cdf(np.diag(var), u, 1024, 8, 5)
    ref = np.prod([special.ndtr(u[i] / math.sqrt(var[i])) for i in range(5)])
    assert p == pytest.approx(ref, rel=1e-13)
    assert rse < 1e-13


@pytest.mark.parametrize("rho", [-0.9, -0.3, 0.0, 0.5, 0.95])
def test_bivariate_orthant(rho):
    S = np.array([[1.0, rho], [rho, 1.0]])
    p, rse = O.genz_cdf(S, [0.0, 0.0], 2048, 16, 1)
    ref = 0.25 + math.asin(rho) / (2 * math.pi)
    assert _within(p, rse, ref)


def test_trivariate_orthant():
    S = np.array([[1.0, 0.3, -0.2], [0.3, 1.0, 0.6], [-0.2, 0.6, 1.0]])
    p, rse = O.genz_cdf(S, np.zeros(3), 4096, 16, 2)
    ref = 0.125 + (math.asin(0.3) + math.asin(-0.2) + math.asin(0.6)) / (4 * math.pi)
    assert _within(p, rse, ref)


@pytest.mark.parametrize("D", [2, 3, 5, 8, 12, 20])
def test_equicorrelated_half_orthant(D):
    S = np.full((D, D), 0.5) + 0.5 * np.eye(D)
    p, rse = O.genz_cdf(S, np.zeros(D), 4096, 16, D)
    assert _within(p, rse, 1.0 / (D + 1), floor=1e-9)


def _bvn_quad(a, b, rho):
    """P(X < a, Y < b) = int_{-inf}^a phi(x) Phi((b - rho x)/sqrt(1-rho^2)) dx."""
    s = math.sqrt(1 - rho * rho)
    f = lambda x: math.exp(-0.5 * x * x) / math.sqrt(2 * math.pi) * special.ndtr((b - rho * x) / s)
    v, _ = integrate.quad(f, -np.inf, a, epsabs=1e-14, epsrel=1e-13, limit=200)
    return v


@pytest.mark.parametrize("a,b,rho", [(0.5, -0.3, 0.7), (-1.5, 2.0, -0.4), (1.0, 1.0, 0.95)])
def test_bivariate_general_vs_quadrature(a, b, rho):
    S = np.array([[1.0, rho], [rho, 1.0]])
    p, rse = O.genz_cdf(S, [a, b], 4096, 16, 3)
    assert _within(p, rse, _bvn_quad(a, b, rho))


def test_convergence_in_n():
    rho = 0.6
    S = np.array([[1.0, rho], [rho, 1.0]])
    ref = _bvn_quad(0.2, 0.7, rho)
    errs = [abs(O.genz_cdf(S, [0.2, 0.7], N, 16, 9)[0] - ref) for N in (64, 1024, 8192)]
    assert errs[2] < errs[0]


@pytest.mark.parametrize("D", [3, 4, 6])
def test_brute_force_monte_carlo(D):
    s = inputs.uniform_sites(D, 30 + D)
    Sig = O.cov_matrix(s, O.COV_EXPONENTIAL, 1.0, 0.3)
    u = inputs.rng(30 + D, 1).normal(0.3, 0.5, size=D)
    p, rse = O.genz_cdf(Sig, u, 4096, 16, 4)
    L = np.linalg.cholesky(Sig)
    r = inputs.rng(777, D)
    n_total, hits = 0, 0
    for _ in range(10):
        z = r.standard_normal((2_000_000, D))
        x = z @ L.T
        hits += int(np.all(x < u, axis=1).sum())
        n_total += z.shape[0]
    mc = hits / n_total
    se_mc = math.sqrt(mc * (1 - mc) / n_total)
    assert abs(p - mc) <= 4 * math.sqrt((p * rse) ** 2 + se_mc ** 2)


def test_not_pd_block():
    S = np.array([[1.0, 1.0], [1.0, 1.0]])
    with pytest.raises(O.OracleError) as e:
        O.genz_cdf(S, [0.0, 0.0], 64, 2, 0)
    assert e.value.status == O.ERR_NOT_PD
