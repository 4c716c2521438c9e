"""GPU parity of the censored likelihood G_I (Sec. 4, Eq. model05): the
conditional law of the censored sites on the device (V = L^-1 Sigma_Ic,
thresholds x_c - V w) and the Vecchia terms with the low-rank-corrected
covariance, against the oracle (LAPACK solves, explicit conditional
covariance): FP64 <= 1e-10 relative, mixed <= 1e-4 max(1, |log G_I|)."""
import numpy as np
import pytest

import oracle as O
from paper_2007_15195_gb300 import binding as B
from paper_2007_15195_gb300 import inputs

from _prep import mixed_tol

pytestmark = pytest.mark.gpu

COV = (O.COV_EXPONENTIAL, 1.0, 0.3, 0.5, 0.0)


@pytest.fixture(scope="module")
def ctx():
    c = B.Context(0)
    yield c
    c.close()


def _split(D, k, seed, m, cov=COV):
    prob = inputs.small_random(D, seed, m=m, cov=cov)
    perm = O.order(prob.sites, O.ORDER_MAXMIN)
    s, x = prob.sites[perm], prob.u[perm]
    rng = np.random.default_rng(seed)
    obs = np.sort(rng.choice(D, size=k, replace=False))
    cen = np.setdiff1d(np.arange(D), obs)
    return (np.ascontiguousarray(s[cen]), np.ascontiguousarray(x[cen]), np.ascontiguousarray(s[obs]),
            np.ascontiguousarray(x[obs] + 1.0))


def _check(got, ref, prec):
    tol = 1e-10 * abs(ref) if prec == B.FP64 else mixed_tol(ref)
    assert abs(got - ref) <= tol, (got, ref, prec)


@pytest.mark.parametrize("prec", [B.FP64, B.MIXED])
@pytest.mark.parametrize("D,k,m,n_nodes", [(120, 8, 10, 0), (120, 8, 10, 6), (200, 40, 20, 4), (90, 3, 40, 0),
                                            (400, 150, 10, 0)])  # 5 blocks of Sigma_II: the two-stream factor
def test_censored_against_oracle(ctx, prec, D, k, m, n_nodes):
    sc, xc, si, xi = _split(D, k, 10 + k, m)
    nbr = B.vecchia_neighbors(ctx, sc, m)
    ref_nbr = O.neighbors(sc, m)
    assert np.array_equal(nbr, ref_nbr)
    ref = O.censored_log_cdf(sc, ref_nbr, m, si, COV, xc, xi, 512, 4, 7, 0.6, 1.0, n_nodes)
    lg, se = B.vecchia_censored_log_cdf(ctx, sc, nbr, m, si, COV, xc, xi, 512, 4, seed=7, beta=0.6, gamma=1.0,
                                        n_nodes=n_nodes, precision=prec)
    _check(lg, ref, prec)
    assert se >= 0


def test_censored_anisotropic_fp64(ctx):
    cov = (B.COV_ANISO_EXP, 1.2, 0.25, 0.5, 0.02, 0.4, 1.8)
    sc, xc, si, xi = _split(100, 6, 3, 8, cov=cov)
    nbr = O.neighbors(sc, 8)
    ref = O.censored_log_cdf(sc, nbr, 8, si, cov, xc, xi, 256, 4, 2, n_nodes=0)
    lg, _ = B.vecchia_censored_log_cdf(ctx, sc, nbr, 8, si, cov, xc, xi, 256, 4, seed=2, n_nodes=0,
                                       precision=B.FP64)
    _check(lg, ref, B.FP64)


def test_nothing_observed_is_the_mixture(ctx):
    sc, xc, _, _ = _split(80, 0, 5, 6)
    nbr = B.vecchia_neighbors(ctx, sc, 6)
    a = B.vecchia_censored_log_cdf(ctx, sc, nbr, 6, np.zeros((0, 2)), COV, xc, np.zeros(0), 256, 4, seed=1,
                                   n_nodes=5)
    b = B.vecchia_mixture_log_cdf(ctx, sc, nbr, 6, COV, xc, 256, 4, 1, n_nodes=5)
    assert a == b


def test_nothing_censored_is_the_density(ctx):
    _, _, si, xi = _split(30, 30, 6, 0)
    ref = O.censored_log_cdf(np.zeros((0, 2)), np.zeros((0, 1), np.int32), 1, si, COV, np.zeros(0), xi, 64, 2, 0,
                             0.5, 1.0, 8)
    lg, se = B.vecchia_censored_log_cdf(ctx, np.zeros((0, 2)), None, 0, si, COV, np.zeros(0), xi, 64, 2, n_nodes=8)
    assert lg == pytest.approx(ref, rel=1e-12) and se == 0.0


def test_host_and_device_inputs_agree(ctx):
    import torch
    sc, xc, si, xi = _split(150, 12, 8, 10)
    nbr = B.vecchia_neighbors(ctx, sc, 10)
    a = B.vecchia_censored_log_cdf(ctx, sc, nbr, 10, si, COV, xc, xi, 512, 4, seed=3, n_nodes=3)
    t = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()
    b = B.vecchia_censored_log_cdf(ctx, t(sc), t(nbr), 10, t(si), COV, t(xc), t(xi), 512, 4, seed=3, n_nodes=3)
    assert a == b


def test_singular_observed_covariance(ctx):
    sc, xc, si, xi = _split(60, 5, 9, 4)
    si[1] = si[0]
    with pytest.raises(B.VecchiaError) as e:
        B.vecchia_censored_log_cdf(ctx, sc, O.neighbors(sc, 4), 4, si, COV, xc, xi, 256, 4, n_nodes=0,
                                   precision=B.FP64)
    assert e.value.status == B.ERR_NOT_PD and B.vecchia_last_error_site(ctx) == 1
