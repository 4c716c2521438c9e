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
    # near Phi = 1/2 the exponent a ~ -2 carries a few FP32 roundings of its
    # Horner sum (~2 ulp of 2, 1.6e-7 relative after ln 2) on top of the fit:
    # about 4 ulp of 1/2 in absolute terms
    assert np.max(np.abs(e - ref)) < 2.5e-7


KZS = np.sqrt(np.log2(np.e) / 2.0)  # the fast mixed step carries kZs z


def test_phi_scaled_form_of_the_fast_step(ctx):
    """Phi from zs = kZs z (one fma for the exponent): the same accuracy as
    the unscaled form, for z = zs / kZs."""
    zs = np.linspace(-9.0, 9.0, 200001) * KZS
    e, zf = _run(ctx, 5, zs)
    ec, _ = _run(ctx, 6, zs)
    x = zf / KZS
    ref, refc = special.ndtr(x), special.ndtr(-x)
    small = np.where(x < 0, e, ec)
    small_ref = np.where(x < 0, ref, refc)
    a = 0.5 * x * x * np.log2(np.e)
    bound = 8e-7 + 1.2e-7 * np.maximum(a, 1.0)
    assert np.all(np.abs(small - small_ref) / small_ref < bound)
    assert np.max(np.abs(e - ref)) < 2.5e-7
    assert np.all(e + ec == pytest.approx(1.0, abs=1.2e-7))


def test_quantile_scaled_form_of_the_fast_step(ctx):
    """Phi^{-1} from 16 p and 16 q, the central polynomial in log2(256 p q)."""
    p = np.concatenate([10.0 ** -np.linspace(37.5, 0.31, 20001), np.linspace(0.49, 0.999999, 20001)])
    y, pf = _run(ctx, 7, p)
    qf = (1.0 - pf.astype(np.float32)).astype(np.float64)
    ref = np.where(pf <= 0.5, special.ndtri(pf), -special.ndtri(qf))
    err = np.abs(y - ref) / np.maximum(1.0, np.abs(ref))
    assert np.max(err) < 2e-6
    # the central piece (p q > 2^-14.3) on its own: fit and FP32 evaluation
    central = pf * qf > 2.0 ** -14.3
    assert np.max(err[central]) < 8e-7


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


# ---- FP64 forms of the FP64 path (vecchia_eval_special64) ----

def _run64(ctx, which, x):
    import torch
    xs = torch.tensor(np.asarray(x, dtype=np.float64), device="cuda")
    return B.vecchia_eval_special64(ctx, which, xs).cpu().numpy()


def test_phi64_relative_error_of_the_smaller_tail(ctx):
    # Phi(-a) = exp(-a^2/2) R(a): R piecewise (fit ~5e-16), the exponential
    # table-driven with a^2/2 carried exactly; a few 1e-16 overall.  The
    # reference is scipy's ndtr, which rounds the square of x/sqrt(2) before
    # exponentiating it: its own relative error grows like 2^-53 a^2 in the
    # tail, which the bound allows for.
    x = np.concatenate([np.linspace(-37.5, 37.5, 400001), [0.0, -1e-300, 1e-300, -0.125, 0.125]])
    e = _run64(ctx, 0, x)
    ec = _run64(ctx, 1, x)
    small = np.where(x < 0, e, ec)
    small_ref = special.ndtr(-np.abs(x))
    rel = np.abs(small - small_ref) / small_ref
    bound = 2e-15 + 4.5e-16 * x * x
    assert np.all(rel < bound), (np.max(rel / bound), x[np.argmax(rel / bound)])
    core = np.abs(x) <= 2.0
    assert np.max(rel[core]) < 4e-15
    assert np.max(np.abs(e - special.ndtr(x))) < 4.5e-16  # two units in the last place below 1
    assert np.all(e + ec == pytest.approx(1.0, abs=2e-16))


def test_phi64_below_the_normal_range(ctx):
    # Phi(x) between ~6e-323 and 2^-1022 (subnormal results).  scipy's ndtr
    # flushes to 0 below x ~ -37.7; libm's erfc (the oracle's Phi) does not.
    import oracle as O
    x = np.linspace(-38.4, -37.6, 801)
    e = _run64(ctx, 0, x)
    ref = np.array([O.Phi(v) for v in x])
    assert np.all(ref > 0)
    assert np.all(np.abs(e - ref) <= 1e-12 * ref + 1e-323)


def test_quantile64_from_either_tail(ctx):
    # one Halley step from the FP32 first guess: ~1e-15 relative
    p = np.concatenate([10.0 ** -np.linspace(300.0, 0.31, 40001), np.linspace(0.49, 0.5, 1001)])
    y = _run64(ctx, 2, p)
    ref = special.ndtri(p)
    err = np.abs(y - ref) / np.maximum(np.abs(ref), 1e-300)
    assert np.max(err[p < 0.4]) < 2e-14, (np.max(err), p[np.argmax(err)])
    assert np.max(np.abs(y - ref)[p >= 0.4]) < 1e-15
    yu = _run64(ctx, 3, p)  # Phi^{-1}(1 - p) from q = p
    erru = np.abs(yu + ref) / np.maximum(np.abs(ref), 1e-300)
    assert np.max(erru[p < 0.4]) < 2e-14
    assert np.max(np.abs(yu + ref)[p >= 0.4]) < 1e-15


def test_quantile64_clamps_at_2_pow_minus_1000(ctx):
    y = _run64(ctx, 2, np.array([0.0, 1e-310, 2.0 ** -1000, 2.0 ** -999]))
    ref = special.ndtri(np.array([2.0 ** -1000, 2.0 ** -1000, 2.0 ** -1000, 2.0 ** -999]))
    assert np.max(np.abs(y - ref) / np.abs(ref)) < 2e-14
