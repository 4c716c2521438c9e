"""Pins of the oracle's scale-mixture CDF G(x) = int Phi_D(x/r) dF_R(r)
(Sec. 4, Eq. model01-model03), by quadrature over v = F_R(r)."""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O
from paper_2007_15195_gb300 import inputs


def _prep(D, seed, m):
    prob = inputs.small_random(D, seed, m=m, N=256, S=4)
    perm = O.order(prob.sites, O.ORDER_MAXMIN)
    s, u = prob.sites[perm], prob.u[perm]
    return prob, s, u, O.neighbors(s, m)


def test_mixing_distribution_inverse():
    for beta, gamma in [(0.5, 1.0), (2.0, 0.3), (0.0, 2.0)]:
        for v in [0.0, 0.1, 0.5, 0.99]:
            r = O.mixing_quantile(v, beta, gamma)
            F = (1 - math.exp(-gamma * (r ** beta - 1) / beta)) if beta > 0 else 1 - r ** (-gamma)
            assert F == pytest.approx(v, abs=1e-13)
            assert r >= 1.0


def test_orthant_is_scale_free():
    """x = 0: Phi_D(0/r) = Phi_D(0) for every r, so G = Phi_D(0)."""
    prob, s, u, nbr = _prep(40, 1, 5)
    x = np.zeros(40)
    lg = O.mixture_log_cdf(s, nbr, 5, prob.cov, x, 256, 4, 0, 0.7, 1.3, 12)
    lp, _ = O.log_cdf(s, nbr, 5, prob.cov, x, 256, 4, 0)
    assert lg == pytest.approx(lp, abs=1e-12)


def test_nodes_integrate_polynomials_in_v_exactly():
    """v^k (1-t)^3 is a polynomial of degree 4k+3 in t: exact for 4k+3 <= 2n-1."""
    v, w = O.mixture_nodes(12)
    assert np.all((v > 0) & (v < 1)) and np.all(w > 0)
    for k in range(6):
        assert np.sum(w * v ** k) == pytest.approx(1.0 / (k + 1), abs=1e-14)


def _fR(beta, gamma):
    if beta > 0:
        return lambda r: gamma * r ** (beta - 1) * math.exp(-gamma * (r ** beta - 1) / beta)
    return lambda r: gamma * r ** (-gamma - 1)


@pytest.mark.parametrize("beta,gamma,xv", [(0.8, 1.5, 0.9), (0.5, 1.0, -2.0), (2.0, 1.0, -4.0),
                                           (0.2, 1.0, 1.5), (0.0, 1.0, -2.0)])
def test_one_dimension_against_quadrature(beta, gamma, xv):
    """D = 1: G(x) = int_1^inf Phi(x/r) f_R(r) dr by adaptive quadrature in r."""
    s = np.array([[0.3, 0.3]])
    lg = O.mixture_log_cdf(s, np.zeros((1, 0), np.int32), 0, (0, 1.0, 0.2, 0.5, 0.0), np.array([xv]), 64, 2, 0,
                           beta, gamma, 32)
    ref, _ = integrate.quad(lambda r: special.ndtr(xv / r) * _fR(beta, gamma)(r), 1.0, np.inf,
                            epsabs=1e-15, epsrel=1e-13, limit=500)
    assert lg == pytest.approx(math.log(ref), abs=1e-9)


def test_independent_components_against_quadrature():
    """Three sites far apart at a tiny range: Sigma = I, so the Vecchia terms are
    exact and G(x) = int prod_i Phi(x_i/r) f_R(r) dr."""
    s = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    x = np.array([0.4, -1.1, 2.0])
    nbr = O.neighbors(s, 2)
    beta, gamma = 0.7, 1.0
    lg = O.mixture_log_cdf(s, nbr, 2, (0, 1.0, 1e-3, 0.5, 0.0), x, 64, 2, 0, beta, gamma, 32)
    f = lambda r: np.prod(special.ndtr(x / r)) * _fR(beta, gamma)(r)
    ref, _ = integrate.quad(f, 1.0, np.inf, epsabs=1e-15, epsrel=1e-13, limit=500)
    assert lg == pytest.approx(math.log(ref), abs=1e-9)


def test_degenerate_mixing_gives_the_gaussian_cdf():
    """beta = 0 with a huge gamma: R is 1 almost surely, so G = Phi_D."""
    prob, s, u, nbr = _prep(30, 2, 6)
    lg = O.mixture_log_cdf(s, nbr, 6, prob.cov, u, 256, 4, 0, 0.0, 1e7, 8)
    lp, _ = O.log_cdf(s, nbr, 6, prob.cov, u, 256, 4, 0)
    assert lg == pytest.approx(lp, abs=1e-5)
