"""Pins of the oracle's censored likelihood G_I (Sec. 4, Eq. model05).

  - Vecchia from an explicit covariance matrix equals the site-based path bit
    for bit (the blocks are the same entries);
  - nothing observed (k = 0): G_I is G of Eq. (model03) (mixture) or Phi_D;
  - nothing censored (c = 0), R = 1: the Gaussian log-density (scipy);
  - one observed, one censored, R = 1: phi(x_1) Phi((x_2 - rho x_1)/sqrt(1 - rho^2));
    with the mixing law: a 1-D quadrature in r of the same product;
  - the conditional law: mean and covariance against the joint-Gaussian
    identities via a brute-force check on a 3-site example (Monte Carlo of
    the conditional CDF).
"""
import math

import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle as O
from paper_2007_15195_gb300 import inputs

COV = (O.COV_EXPONENTIAL, 1.0, 0.3, 0.5, 0.0)


def _split(D, k, seed, m):
    prob = inputs.small_random(D, seed, m=m, cov=COV)
    perm = O.order(prob.sites, O.ORDER_MAXMIN)
    s, x = prob.sites[perm], prob.u[perm]
    rng = np.random.default_rng(seed)
    obs = np.sort(rng.choice(D, size=k, replace=False))
    cen = np.setdiff1d(np.arange(D), obs)
    sc, xc = s[cen], x[cen]
    return sc, xc, s[obs], x[obs] + 1.0, O.neighbors(sc, m)


def test_vecchia_from_matrix_equals_site_path():
    prob = inputs.small_random(60, 4, m=6, cov=COV)
    perm = O.order(prob.sites, O.ORDER_MAXMIN)
    s, u = prob.sites[perm], prob.u[perm]
    nbr = O.neighbors(s, 6)
    a = O.vecchia_from_matrix(O.cov_matrix(s, *COV[:3]), nbr, 6, u, 256, 4, 2)
    b = O.log_cdf(s, nbr, 6, COV, u, 256, 4, 2)
    assert a == b


@pytest.mark.parametrize("n_nodes", [0, 8])
def test_nothing_observed_is_the_cdf(n_nodes):
    sc, xc, _, _, nbr = _split(40, 0, 3, 5)
    g = O.censored_log_cdf(sc, nbr, 5, np.zeros((0, 2)), COV, xc, np.zeros(0), 256, 4, 1, 0.7, 1.0, n_nodes)
    ref = (O.log_cdf(sc, nbr, 5, COV, xc, 256, 4, 1)[0] if n_nodes == 0
           else O.mixture_log_cdf(sc, nbr, 5, COV, xc, 256, 4, 1, 0.7, 1.0, n_nodes))
    assert g == pytest.approx(ref, abs=1e-12)


def test_nothing_censored_is_the_gaussian_density():
    s = inputs.uniform_sites(7, 9)
    x = np.linspace(-0.5, 1.2, 7)
    g = O.censored_log_cdf(np.zeros((0, 2)), np.zeros((0, 3), np.int32), 3, s, COV, np.zeros(0), x, 64, 2, 0,
                           n_nodes=0)
    ref = stats.multivariate_normal(np.zeros(7), O.cov_matrix(s, *COV[:3])).logpdf(x)
    assert g == pytest.approx(ref, abs=1e-10)


def _two_site(rho_h):
    s = np.array([[0.0, 0.0], [rho_h, 0.0]])
    return s, math.exp(-rho_h / 0.3)


def test_one_observed_one_censored_gaussian():
    s, rho = _two_site(0.2)
    x1, x2 = 0.4, -0.3
    g = O.censored_log_cdf(s[1:], np.zeros((1, 1), np.int32) - 1, 1, s[:1], COV, np.array([x2]),
                           np.array([x1]), 64, 2, 0, n_nodes=0)
    ref = math.log(special.ndtr((x2 - rho * x1) / math.sqrt(1 - rho * rho)) * stats.norm.pdf(x1))
    assert g == pytest.approx(ref, abs=1e-13)


def test_one_observed_one_censored_mixture_against_quadrature():
    s, rho = _two_site(0.15)
    x1, x2, beta, gamma = 0.8, 0.2, 0.6, 1.0
    g = O.censored_log_cdf(s[1:], np.zeros((1, 1), np.int32) - 1, 1, s[:1], COV, np.array([x2]),
                           np.array([x1]), 64, 2, 0, beta, gamma, 32)
    fR = lambda r: gamma * r ** (beta - 1) * math.exp(-gamma * (r ** beta - 1) / beta)
    f = lambda r: (special.ndtr((x2 - rho * x1) / (r * math.sqrt(1 - rho * rho))) * stats.norm.pdf(x1 / r) / r
                   * fR(r))
    ref, _ = integrate.quad(f, 1.0, np.inf, epsabs=1e-15, epsrel=1e-13, limit=500)
    assert g == pytest.approx(math.log(ref), abs=1e-8)


def test_conditional_law_by_monte_carlo():
    """Three sites, one observed: Phi_2 of the conditional law (telescoping
    Vecchia with m = 1) against a Monte Carlo of X_c | X_I = x_I drawn from the
    joint Gaussian by rejection-free conditioning on a fine slab."""
    s = np.array([[0.0, 0.0], [0.1, 0.05], [0.25, 0.0]])
    Sig = O.cov_matrix(s, *COV[:3])
    x = np.array([0.3, 0.2, 0.5])
    I, cidx = [1], [0, 2]
    g = O.censored_log_cdf(s[cidx], np.array([[-1], [0]], np.int32), 1, s[I], COV, x[cidx], x[I], 4096, 16, 5,
                           n_nodes=0)
    # independent evaluation: conditional mean/cov from the joint Gaussian by
    # regression on samples, then the bivariate CDF by sampling
    rng = np.random.default_rng(0)
    Z = rng.multivariate_normal(np.zeros(3), Sig, size=400_000)
    A = np.linalg.lstsq(np.c_[Z[:, I]], Z[:, cidx], rcond=None)[0]       # regression coefficients
    resid = Z[:, cidx] - Z[:, I] @ A
    mu = (x[I] @ A)
    C = np.cov(resid.T)
    W = rng.multivariate_normal(mu, C, size=400_000)
    p = np.mean(np.all(W < x[cidx], axis=1))
    ref = math.log(p) + stats.norm.logpdf(x[1], scale=math.sqrt(Sig[1, 1]))
    assert g == pytest.approx(ref, abs=0.02)
