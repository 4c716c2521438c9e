"""The FP32 normal CDF and quantile of the mixed path (own fitted forms),
evaluated on the GPU through vecchia_eval_special, against scipy's FP64
ndtr / ndtri.  These are the per-coordinate maps of Genz's separation of
variables (Sec. 2.2)."""
import numpy as np
import pytest
from scipy import special

from paper_2007_15195_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    c = B.Context(0)
    yield c
    c.close()


def _run(ctx, which, x):
    import torch
    xs = torch.tensor(np.asarray(x, dtype=np.float32), device="cuda")
    return B.vecchia_eval_special(ctx, which, xs).cpu().numpy().astype(np.float64), \
        xs.cpu().numpy().astype(np.float64)


def test_phi_relative_error_of_the_smaller_tail(ctx):
    x = np.linspace(-9.0, 9.0, 200001)
    e, xf = _run(ctx, 0, x)
    ec, _ = _run(ctx, 1, x)
    ref = special.ndtr(xf)
    refc = special.ndtr(-xf)
    small = np.where(xf < 0, e, ec)
    small_ref = np.where(xf < 0, ref, refc)
    # Phi(-|x|) = t 2^a with a ~ -x^2 log2(e)/2: the FP32 rounding of a moves
    # the result by ~|a| 2^-24 ln 2 relative, on top of ~5e-7 from the fit and the
    # approximate reciprocal and exponential.
    a = 0.5 * xf * xf * np.log2(np.e)
    bound = 8e-7 + 1.2e-7 * np.maximum(a, 1.0)
    assert np.all(np.abs(small - small_ref) / small_ref < bound)
    assert np.max(np.abs(e - ref)) < 2e-7


def test_log2_phi_far_tail(ctx):
    x = np.linspace(-37.5, -9.01, 50001)
    l2, xf = _run(ctx, 2, x)
    ref = special.log_ndtr(xf) / np.log(2.0)
    assert np.all(np.isfinite(l2))
    assert np.max(np.abs(l2 - ref) / np.abs(ref)) < 1e-6


def test_quantile_lower_and_upper(ctx):
    p = np.concatenate([10.0 ** -np.linspace(37.5, 0.31, 20001), np.linspace(0.49, 0.999999, 20001)])
    y, pf = _run(ctx, 3, p)
    qf = (1.0 - pf.astype(np.float32)).astype(np.float64)  # the kernel sees q = 1 - p in FP32
    ref = np.where(pf <= 0.5, special.ndtri(pf), -special.ndtri(qf))
    err = np.abs(y - ref) / np.maximum(1.0, np.abs(ref))
    assert np.max(err) < 2e-6


def test_quantile_from_log2(ctx):
    lr2 = np.linspace(-1000.0, -64.0, 50001)
    y, lf = _run(ctx, 4, lr2)
    ref = special.ndtri(np.exp2(lf))
    assert np.max(np.abs(y - ref) / np.abs(ref)) < 1e-6
