"""The bounded device waits of the tensor-core full Genz kernel.

Its point warps wait on mbarriers for the accumulators the copy lane's MMAs
fill; every wait is bounded by the global timer, and a wait that runs out
makes the kernel record a timeout, drain what it issued, free its tensor
memory and return, so the call reports VECCHIA_ERR_TIMEOUT and the context
stays usable.  The test makes a wait run out without any fault: a short wait
limit, and the copy lane told to issue nothing, so the accumulator barrier the
point warps wait on is one that nothing completes (no copy or MMA in flight).
The next call, with the default restored, must still match the oracle.
"""
import numpy as np
import pytest

import oracle as O
from paper_2007_15195_gb300 import binding as B
from paper_2007_15195_gb300 import inputs

from _prep import mixed_tol

pytestmark = pytest.mark.gpu


def test_full_genz_wait_runs_out_and_context_recovers():
    prob = inputs.small_random(200, 41, m=0, u_mean=0.3)
    perm = O.order(prob.sites, O.ORDER_MAXMIN)
    s = np.ascontiguousarray(prob.sites[perm])
    u = np.ascontiguousarray(prob.u[perm])
    N, S = 512, 4
    ref, _ = O.full_genz(s, prob.cov, u, N, S, 5)
    with B.Context(0) as ctx:
        B.vecchia_set_full_genz_wait(ctx, limit_ns=1_000_000, withhold=True)  # 1 ms, nothing issued
        with pytest.raises(B.VecchiaError) as e:
            B.vecchia_full_genz(ctx, s, prob.cov, u, N, S, seed=5, precision=B.MIXED)
        assert e.value.status == B.ERR_TIMEOUT
        B.vecchia_set_full_genz_wait(ctx, 0, False)
        lp, _ = B.vecchia_full_genz(ctx, s, prob.cov, u, N, S, seed=5, precision=B.MIXED)
        assert abs(lp - ref) <= mixed_tol(ref), (lp, ref)
        # the FP64 path has no device waits: unaffected either way
        B.vecchia_set_full_genz_wait(ctx, limit_ns=1_000_000, withhold=True)
        lp64, _ = B.vecchia_full_genz(ctx, s, prob.cov, u, N, S, seed=5, precision=B.FP64)
        assert abs(lp64 - ref) <= 1e-10 * abs(ref)
