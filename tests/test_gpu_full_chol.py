"""The Cholesky factor behind the full D-dimensional estimate (Sec. 2.2: the
factor of the whole covariance that Genz's recursion runs on), through
vecchia_full_cholesky: the FP64 blocked factor and the mixed path's trailing
updates on the tensor cores (bf16 digit slices, exact FP32 accumulation, FP64
recombination), each against LAPACK's Cholesky of the oracle's covariance.

Two FP64 factorizations of one matrix differ by their roundings amplified by
its conditioning: a one-ulp perturbation of the 50x50-grid covariance
(condition 6.8e4) moves its factor by 2.5e-14 of its largest entry, the
better-conditioned uniform sets by ~2e-15; 1e-12 leaves a margin of 40 and
would catch an inexact accumulation (FP32 rounding of the digit sums: ~1e-7)."""
import numpy as np
import pytest

import oracle as O
from paper_2007_15195_gb300 import binding as B, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch  # noqa: F401
    c = B.Context(0)
    yield c
    c.close()


def _case(kind, D):
    if kind == "grid50":
        s = inputs.grid50(m=20).sites
        cov = (B.COV_MATERN, 1.0, 0.1, 1.5, 0.0)
    else:
        s = inputs.uniform_sites(D, 5)
        cov = (B.COV_EXPONENTIAL, 1.0, 0.1, 0.5, 0.0)
    return np.ascontiguousarray(s[O.order(s, 0)]), cov


@pytest.mark.parametrize("kind,D", [("grid50", 2500), ("u", 1000), ("u", 777), ("u", 100), ("u", 64), ("u", 33)])
def test_factor_against_lapack(ctx, kind, D):
    s, cov = _case(kind, D)
    S = O.cov_matrix(s, *cov)
    Lref = np.linalg.cholesky(S)
    scale = np.max(np.abs(Lref))
    L64 = B.vecchia_full_cholesky(ctx, s, cov, B.FP64)
    Lmx = B.vecchia_full_cholesky(ctx, s, cov, B.MIXED)
    for L in (L64, Lmx):
        assert np.all(np.triu(L, 1) == 0.0)
        assert np.max(np.abs(L - Lref)) / scale < 1e-12
    assert np.max(np.abs(Lmx - L64)) / scale < 1e-12


def test_factor_from_device_arrays(ctx):
    import torch
    s, cov = _case("u", 500)
    out = torch.empty((500, 500), dtype=torch.float64, device="cuda")
    B.vecchia_full_cholesky(ctx, torch.from_numpy(s).cuda(), cov, B.MIXED, out=out)
    Lh = B.vecchia_full_cholesky(ctx, s, cov, B.MIXED)
    assert np.array_equal(out.cpu().numpy(), Lh)


def test_singular_covariance_reports_the_row(ctx):
    """Sites 0 and 40 equal (different blocks of 32 columns), no nugget: the
    pivot of row 40 vanishes up to rounding.  A zero or negative one is
    reported (or, if it came out positive, a later row that its rounding-size
    pivot spoils); a positive one leaves L_40,40 of rounding size."""
    s, cov = _case("u", 200)
    s[40] = s[0]
    for prec in (B.FP64, B.MIXED):
        try:
            L = B.vecchia_full_cholesky(ctx, s, cov, prec)
        except B.VecchiaError as e:
            assert e.status == B.ERR_NOT_PD and B.vecchia_last_error_site(ctx) >= 40
        else:
            assert abs(L[40, 40]) < 1e-6
