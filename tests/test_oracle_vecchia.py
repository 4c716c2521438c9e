"""Pins of the oracle's Vecchia log-CDF (Eq. vecchia-cdf, Sec. 2.2).

  - m = 0: every term is the univariate Phi(u_i / sigma) exactly.
  - m = D - 1: Eq. (vecchia-cdf) is the telescoping product of Eq.
    (cascading-conditional-cdf); with common lattice points and shifts the
    estimate equals the log of the full D-dimensional Genz estimate up to the
    rounding of the final sum, and the standard error equals its relative SE.
  - independence: every recursion sample is the product of univariate Phi.
  - scale invariance: (sigma^2, u) and (1, u / sigma) give the same result.
  - D = 2: the single term is the bivariate CDF over Phi(u_1) (1-D quadrature).
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O
from paper_2007_15195_gb300 import inputs


def _prep(prob):
    perm = O.order(prob.sites, {"xy": O.ORDER_XY, "maxmin": O.ORDER_MAXMIN,
                                "identity": O.ORDER_IDENTITY}[prob.order])
    s = prob.sites[perm]
    u = prob.u[perm]
    nbr = O.neighbors(s, prob.m)
    return s, u, nbr


def test_m0_is_sum_of_univariate():
    prob = inputs.small_random(40, 1, m=0, cov=(O.COV_MATERN, 2.0, 0.2, 1.5, 0.0))
    s, u, nbr = _prep(prob)
    lp, se = O.log_cdf(s, nbr, 0, prob.cov, u, 256, 4, 0)
    ref = sum(math.log(special.ndtr(x / math.sqrt(2.0))) for x in u)
    assert lp == pytest.approx(ref, rel=1e-13)
    assert se == 0.0


@pytest.mark.parametrize("D,N", [(2, 1024), (5, 1024), (17, 512), (60, 256), (200, 64)])
def test_m_full_is_telescoping_identity(D, N):
    prob = inputs.small_random(D, D, m=D - 1, cov=(O.COV_EXPONENTIAL, 1.0, 0.3, 0.5, 0.0))
    s, u, nbr = _prep(prob)
    lp_v, se_v = O.log_cdf(s, nbr, D - 1, prob.cov, u, N, 4, 11)
    lp_f, se_f = O.full_genz(s, prob.cov, u, N, 4, 11)
    assert lp_v == pytest.approx(lp_f, rel=1e-12, abs=1e-12)
    assert se_v == pytest.approx(se_f, rel=1e-9, abs=1e-14)


def test_neighbour_sets_with_m_full_are_all_previous():
    s = inputs.uniform_sites(30, 2)
    nbr = O.neighbors(s, 29)
    for i in range(30):
        assert nbr[i, :i].tolist() == list(range(i))


def test_independence_exact_for_any_m():
    prob = inputs.small_random(50, 3, m=8, cov=(O.COV_EXPONENTIAL, 1.0, 1e-6, 0.5, 0.0))
    s, u, nbr = _prep(prob)
    lp, se = O.log_cdf(s, nbr, 8, prob.cov, u, 256, 4, 1)
    ref = sum(math.log(special.ndtr(x)) for x in u)
    assert lp == pytest.approx(ref, rel=1e-12)
    assert se < 1e-12


def test_scale_invariance():
    cov2 = (O.COV_MATERN, 4.0, 0.25, 1.5, 0.0)
    cov1 = (O.COV_MATERN, 1.0, 0.25, 1.5, 0.0)
    prob = inputs.small_random(60, 5, m=6, cov=cov2)
    s, u, nbr = _prep(prob)
    a = O.log_cdf(s, nbr, 6, cov2, u, 512, 4, 2)
    b = O.log_cdf(s, nbr, 6, cov1, u / 2.0, 512, 4, 2)
    assert a[0] == pytest.approx(b[0], rel=1e-12)
    assert a[1] == pytest.approx(b[1], rel=1e-9)


def test_two_sites_vs_quadrature():
    s = np.array([[0.0, 0.0], [0.1, 0.0]])
    rho = math.exp(-0.1 / 0.2)
    u = np.array([0.4, -0.2])
    nbr = O.neighbors(s, 1)
    lp, se = O.log_cdf(s, nbr, 1, (O.COV_EXPONENTIAL, 1.0, 0.2, 0.5, 0.0), u, 4096, 16, 5)
    sd = math.sqrt(1 - rho * rho)
    f = lambda x: math.exp(-0.5 * x * x) / math.sqrt(2 * math.pi) * special.ndtr((u[1] - rho * x) / sd)
    ref, _ = integrate.quad(f, -np.inf, u[0], epsabs=1e-14, epsrel=1e-13)
    assert abs(lp - math.log(ref)) <= 4 * se + 1e-12


def test_terms_sum_and_first_term():
    prob = inputs.grid10()
    s, u, nbr = _prep(prob)
    lp, se, terms = O.log_cdf(s, nbr, 10, prob.cov, u, 256, 4, 0, return_terms=True)
    assert terms[0] == pytest.approx(math.log(0.5), rel=1e-15)  # Phi(0) = 1/2
    assert lp == pytest.approx(terms.sum(), rel=1e-13)
    # each term log P(X_i < u_i | X_N < u_N) is a log-probability
    assert np.all(terms <= 0) and np.all(terms > math.log(0.5) - 1e-12 - 10)


def test_partials_subset_matches_full():
    prob = inputs.small_random(80, 6, m=5)
    s, u, nbr = _prep(prob)
    num, den = O.vecchia_partials(s, nbr, 5, prob.cov, u, 128, 4, 3)
    idx = np.array([0, 1, 5, 6, 40, 79])
    n2, d2 = O.vecchia_partials(s, nbr, 5, prob.cov, u, 128, 4, 3, idx=idx)
    assert np.array_equal(n2, num[idx]) and np.array_equal(d2, den[idx])
    lp, se, terms = O.vecchia_reduce(num, den)
    lp2, se2 = O.log_cdf(s, nbr, 5, prob.cov, u, 128, 4, 3)
    assert lp == lp2 and se == se2


def test_vecchia_increases_toward_full_with_m():
    """Qualitative claim of Sec. 3 (reported, loosely asserted): the Vecchia
    estimate approaches the full estimate as m grows."""
    prob = inputs.small_random(64, 8, m=0, cov=(O.COV_EXPONENTIAL, 1.0, 0.5, 0.5, 0.0), u_mean=0.0,
                               u_sd=0.0, order="xy")
    perm = O.order(prob.sites, O.ORDER_MAXMIN)
    s, u = prob.sites[perm], prob.u[perm]
    full, _ = O.full_genz(s, prob.cov, u, 1024, 8, 1)
    errs = []
    for m in (1, 4, 16, 40):
        nbr = O.neighbors(s, m)
        errs.append(abs(O.log_cdf(s, nbr, m, prob.cov, u, 1024, 8, 1)[0] - full))
    assert errs[-1] < errs[0]


def test_bad_arguments():
    s = inputs.uniform_sites(5, 0)
    nbr = O.neighbors(s, 2)
    with pytest.raises(O.OracleError):
        O.log_cdf(s, nbr, 2, (O.COV_MATERN, 1.0, 0.1, 0.7, 0.0), np.zeros(5), 64, 4, 0)
    with pytest.raises(O.OracleError):
        O.log_cdf(s, nbr, 2, (O.COV_EXPONENTIAL, 1.0, 0.1, 0.5, 0.0), np.zeros(5), 64, 1, 0)
    bad = nbr.copy()
    bad[3, 0] = 3  # not a previous site
    with pytest.raises(O.OracleError):
        O.log_cdf(s, bad, 2, (O.COV_EXPONENTIAL, 1.0, 0.1, 0.5, 0.0), np.zeros(5), 64, 4, 0)


def test_duplicate_sites_not_pd_reports_site():
    s = np.array([[0.0, 0.0], [0.5, 0.5], [0.5, 0.5], [1.0, 0.0]])
    nbr = O.neighbors(s, 2)
    with pytest.raises(O.OracleError) as e:
        O.log_cdf(s, nbr, 2, (O.COV_EXPONENTIAL, 1.0, 0.3, 0.5, 0.0), np.zeros(4), 64, 4, 0)
    assert e.value.status == O.ERR_NOT_PD and e.value.site == 2
