"""The scratch-free entry point vecchia_log_cdf_noalloc against vecchia_log_cdf.

It serves callers that cannot allocate device memory where they evaluate a
log-CDF (under an allocator that owns the device, within a fixed memory budget,
without a context object).  Its scratch lives in a fixed device array that
every call reuses, so the test calls it twice in a row on different problems,
and compares each result with the context-based entry point on the same
device inputs.  Both run the same kernels with the same built-in tile, so the
results must agree bit for bit; the parity tolerances of the other tests only
appear in the failure message, as a diagnostic.  This file sorts last so that
a run stopping at the first failure has run the rest.
"""
import numpy as np
import pytest

from paper_2007_15195_gb300 import binding as B
from paper_2007_15195_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def _mixed_tol(lp):
    return 1e-4 * max(1.0, abs(lp))


def _device_problem(ctx, prob):
    import torch
    perm = B.vecchia_order(ctx, prob.sites, prob.order)
    s = torch.from_numpy(np.ascontiguousarray(prob.sites[perm])).cuda()
    u = torch.from_numpy(np.ascontiguousarray(prob.u[perm])).cuda()
    nbr = B.vecchia_neighbors(ctx, s, prob.m)
    return s, u, nbr


def test_noalloc_matches_log_cdf_on_consecutive_calls():
    import torch
    stream = torch.cuda.current_stream(0).cuda_stream
    with B.Context(0, stream) as ctx:
        B.vecchia_reset_tiles(ctx)
        probs = [inputs.small_random(700, 31, m=20, N=1024, S=8),
                 inputs.grid10(),
                 inputs.small_random(2600, 32, m=9, N=512, S=16)]
        dev = [_device_problem(ctx, p) for p in probs]
        for prec in (B.FP64, B.MIXED):
            for rep in range(2):
                for p, (s, u, nbr) in zip(probs, dev):
                    ref = B.vecchia_log_cdf(ctx, s, nbr, p.m, p.cov, u, p.N, p.S, p.seed + rep, prec)
                    got = B.vecchia_log_cdf_noalloc(0, stream, s, nbr, p.m, p.cov, u, p.N, p.S,
                                                    p.seed + rep, prec)
                    tol = FP64_TOL * abs(ref[0]) if prec == B.FP64 else _mixed_tol(ref[0])
                    diag = "prec %d rep %d: noalloc %r vs log_cdf %r (|d log P| %.3g, parity tol %.3g)" % (
                        prec, rep, got, ref, abs(got[0] - ref[0]), tol)
                    assert got[0] == ref[0], diag
                    assert got[1] == ref[1], diag
        assert torch.cuda.current_device() == 0


def test_noalloc_rejects_host_arrays():
    p = inputs.grid10()
    with B.Context(0) as ctx:
        s, u, nbr = _device_problem(ctx, p)
    with pytest.raises(B.VecchiaError) as e:
        B.vecchia_log_cdf_noalloc(0, None, s.cpu().numpy(), nbr, p.m, p.cov, u, p.N, p.S, 0, B.MIXED)
    assert e.value.status == B.ERR_ARG


def test_noalloc_rejects_problems_beyond_its_array():
    import torch
    D, S, m = 300_000, 16, 5  # 16 D S bytes alone exceed 32 MiB
    s = torch.rand(D, 2, dtype=torch.float64, device="cuda")
    u = torch.zeros(D, dtype=torch.float64, device="cuda")
    nbr = torch.zeros(D, m, dtype=torch.int32, device="cuda")
    with pytest.raises(B.VecchiaError) as e:
        B.vecchia_log_cdf_noalloc(0, None, s, nbr, m, (B.COV_EXPONENTIAL, 1.0, 0.1, 0.5, 0.0), u, 256, S, 0,
                                  B.MIXED)
    assert e.value.status == B.ERR_UNSUPPORTED
