"""C-ABI checks that need no GPU: the library builds and loads, exports every
entry point include/vecchia.h declares, and its host-side logic (lattice,
Philox shifts, ordering, argument checks) agrees with the oracle bit for bit.
"""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2007_15195_gb300 import binding as B
from paper_2007_15195_gb300 import build as libbuild
from paper_2007_15195_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return B.lib()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b(vecchia_\w+)\s*\(", txt, flags=re.M))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["vecchia_create", "vecchia_destroy", "vecchia_order", "vecchia_neighbors",
              "vecchia_log_cdf", "vecchia_log_cdf_batch", "vecchia_lattice", "vecchia_shifts",
              "vecchia_strerror"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (vecchia_\w+)", out))
    missing = _declared() - exported
    assert not missing, missing
    for n in _declared():
        assert hasattr(lib, n)


@pytest.mark.parametrize("N", [2000, 2048, 4096, 8192, 31, 64])
def test_lattice_bit_equal_to_oracle(lib, N):
    assert np.array_equal(B.vecchia_lattice(N, 32), O.lattice(N, 32))


@pytest.mark.parametrize("seed", [0, 1, 12345, (1 << 40) + 7, 2 ** 64 - 1])
def test_shifts_bit_equal_to_oracle(lib, seed):
    assert np.array_equal(B.vecchia_shifts(seed, 16, 31), O.shifts(seed, 16, 31))


def test_order_xy_matches_oracle(lib):
    r = inputs.rng(4, 4)
    s = np.round(r.random((500, 2)) * 16) / 16
    assert np.array_equal(B.vecchia_order(None, s, "xy"), O.order(s, O.ORDER_XY))
    g = inputs.grid_sites(50)
    assert np.array_equal(B.vecchia_order(None, g, "xy"), np.arange(2500))


@pytest.mark.parametrize("D,seed", [(7, 1), (300, 2), (5000, 3)])
def test_order_maxmin_matches_oracle(lib, D, seed):
    s = inputs.uniform_sites(D, seed)
    assert np.array_equal(B.vecchia_order(None, s, "maxmin"), O.order(s, O.ORDER_MAXMIN))


def test_order_maxmin_on_grid_ties(lib):
    s = inputs.grid_sites(20)
    assert np.array_equal(B.vecchia_order(None, s, "maxmin"), O.order(s, O.ORDER_MAXMIN))


def test_order_identity_and_bad_kind(lib):
    s = inputs.uniform_sites(10, 0)
    assert np.array_equal(B.vecchia_order(None, s, "identity"), np.arange(10))
    with pytest.raises(B.VecchiaError) as e:
        B.vecchia_order(None, s, 7)
    assert e.value.status == B.ERR_ARG


def test_strerror(lib):
    assert B.strerror(B.ERR_NOT_PD).startswith("covariance")
    assert B.strerror(12345) == "unknown status"


def test_lattice_and_shift_argument_errors(lib):
    assert lib.vecchia_lattice(0, 4, None) == B.ERR_ARG
    assert lib.vecchia_shifts(C.c_uint64(0), -1, 4, None) == B.ERR_ARG
