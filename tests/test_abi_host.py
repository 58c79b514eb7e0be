"""CPU-side checks of the C ABI: the library loads, exports every declared symbol, and its host-side
(m, s) rule agrees with the oracle's (no GPU compute is called here)."""

import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import select_ms as oracle_select
from oracle.taylor_bound import error_bound as oracle_bound

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(grape_[a-z_0-9]+)\s*\(", txt)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def L():
    from paper_2304_06200_gb300._abi import lib
    return lib()


def test_library_exports_every_declared_symbol(L):
    from paper_2304_06200_gb300._abi import EXPORTED
    declared = _declared_functions()
    assert len(declared) >= 13
    assert sorted(EXPORTED) == declared
    for name in declared:
        assert hasattr(L, name), name
    assert L.grape_abi_version() == 5


def test_status_strings(L):
    for code in range(9):
        assert L.grape_status_string(code)
    assert L.grape_status_string(99) == b"unknown status"


@pytest.mark.parametrize("x", [0.01, 0.7, 2.26, 2.92, 3.47, 7.5, 12.0, 30.3])
@pytest.mark.parametrize("tau", [1e-6, 1e-8, 1e-10, 1e-12])
@pytest.mark.parametrize("sigma", [5, 9])
def test_select_ms_matches_oracle(x, tau, sigma):
    from paper_2304_06200_gb300 import select_ms
    got = select_ms(x, tau, sigma, s_max=200)
    want = oracle_select(x, tau, sigma, s_max=200)
    if got != want:
        # only a pair whose bound sits within rounding of tau may differ
        for pair in (got, want):
            if pair is not None:
                e = oracle_bound(x, pair[0], pair[1], sigma)
                assert abs(e - tau) <= 1e-9 * tau, (got, want, e)
    assert got == want or got is None or want is None or abs(np.prod(got) - np.prod(want)) <= max(got[1], want[1])


@pytest.mark.parametrize("x,m,s", [(0.5, 5, 1), (3.0, 25, 1), (30.0, 31, 6), (30.0, 18, 28), (45.0, 41, 5)])
def test_error_bound_matches_oracle(x, m, s):
    from paper_2304_06200_gb300 import error_bound
    for sigma in (5, 9):
        a = error_bound(x, m, s, sigma)
        b = oracle_bound(x, m, s, sigma)
        assert a == pytest.approx(b, rel=1e-10)


def test_select_ms_infeasible_and_invalid(L):
    from paper_2304_06200_gb300 import select_ms
    assert select_ms(1.0, 1e-17, 5, s_max=64) is None
    m, s = C.c_int32(), C.c_int32()
    assert L.grape_select_ms(-1.0, 1e-8, 5, 0, 60, 100, C.byref(m), C.byref(s)) == 1   # EINVAL


def test_create_rejects_bad_descriptors_before_touching_the_device(L):
    from paper_2304_06200_gb300._abi import GrapeDesc
    d = GrapeDesc()
    h = C.c_void_p()
    assert L.grape_problem_create(None, C.byref(h)) == 1
    d.dim = 0
    assert L.grape_problem_create(C.byref(d), C.byref(h)) == 1
    d.dim, d.n_steps, d.n_states, d.dt, d.tau = 4, 3, 5, 0.1, 1e-8   # n_states > dim
    assert L.grape_problem_create(C.byref(d), C.byref(h)) == 1
    assert not h.value


def test_create_rejects_bad_propagator_choices(L):
    """The eigendecomposition propagator (App. F) is FP64-only and bounded by the shared-memory step matrix."""
    from paper_2304_06200_gb300._abi import GRAPE_FP32_BULK, GRAPE_PROP_EIG, GrapeDesc
    h = C.c_void_p()
    d = GrapeDesc()
    d.dim, d.n_steps, d.n_states, d.dt, d.tau = 4, 3, 1, 0.1, 1e-8
    d.propagator = 2
    assert L.grape_problem_create(C.byref(d), C.byref(h)) == 1
    d.propagator = GRAPE_PROP_EIG
    d.precision = GRAPE_FP32_BULK
    assert L.grape_problem_create(C.byref(d), C.byref(h)) == 1
    assert b"GRAPE_PROP_EIG" in L.grape_last_error()
    d.precision = 0
    d.dim = 97
    assert L.grape_problem_create(C.byref(d), C.byref(h)) == 1
    assert not h.value


@pytest.mark.parametrize("field,value,word", [("backward_mode", 2, b"backward_mode"), ("backward_mode", 4, b"backward_mode"),
                                             ("grad_cluster", 17, b"grad_cluster"), ("block_steps", -1, b"block_steps")])
def test_create_rejects_bad_backward_options(L, field, value, word):
    from paper_2304_06200_gb300._abi import GrapeDesc
    h = C.c_void_p()
    d = GrapeDesc()
    d.dim, d.n_steps, d.n_states, d.dt, d.tau = 4, 3, 1, 0.1, 1e-8
    setattr(d, field, value)
    assert L.grape_problem_create(C.byref(d), C.byref(h)) == 1
    assert word in L.grape_last_error()
    assert not h.value


def test_three_stage_needs_checkpoints(L):
    from paper_2304_06200_gb300._abi import GrapeDesc
    h = C.c_void_p()
    d = GrapeDesc()
    d.dim, d.n_steps, d.n_states, d.dt, d.tau = 4, 3, 1, 0.1, 1e-8
    d.backward_mode, d.ckpt_every = 3, -1
    assert L.grape_problem_create(C.byref(d), C.byref(h)) == 1
    assert b"ckpt_every" in L.grape_last_error()
