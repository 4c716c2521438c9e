"""Shared test helpers: prepare a seeded problem on both sides.

The oracle side orders and searches neighbours with oracle/; the CUDA side
with the library.  Tests assert the two agree, then feed each side its own.
"""
import numpy as np

import oracle as O

ORACLE_ORDER = {"xy": O.ORDER_XY, "maxmin": O.ORDER_MAXMIN, "identity": O.ORDER_IDENTITY}


def oracle_prepare(prob):
    perm = O.order(prob.sites, ORACLE_ORDER[prob.order])
    s = np.ascontiguousarray(prob.sites[perm])
    u = np.ascontiguousarray(prob.u[perm])
    nbr = O.neighbors(s, prob.m) if prob.m > 0 else np.zeros((s.shape[0], 0), np.int32)
    return perm, s, u, nbr


def mixed_tol(log_p):
    """|d log P| <= 1e-4 max(1, |log P|): the mixed-precision bound."""
    return 1e-4 * max(1.0, abs(log_p))
