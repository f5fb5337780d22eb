"""C-ABI library checks that need no GPU: the library loads, exports every
symbol include/sem.h declares, validates arguments on the host, and its host
tables and checkpoint planner agree with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.checkpoint import optimal_advances
from oracle.sem import Grid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1806_01422_gb300 import build, _lib
    build.build()
    return _lib


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "sem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sem_[a-zA-Z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(L):
    names = _declared_symbols()
    assert len(names) >= 15
    lib = L.lib()
    for n in names:
        assert hasattr(lib, n), n
    # and the binding declares a signature for each
    assert set(names) <= set(L._SIGS)


def _create(L, dim, E, N, nu=0.01):
    h = ctypes.c_void_p()
    rc = L.lib().sem_create(dim, E, N, nu, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("dim,E,N,nu", [(0, 2, 3, 0.1), (4, 2, 3, 0.1), (2, 0, 3, 0.1), (2, 2, 0, 0.1),
                                        (2, 2, 16, 0.1), (2, 2, 3, -1.0), (2, 2, 3, float("nan")),
                                        (3, 2, 16, 0.1), (3, 2000, 7, 0.1), (3, 128, 7, 0.1)])
def test_create_rejects_bad_arguments(L, dim, E, N, nu):
    rc, h = _create(L, dim, E, N, nu)
    assert rc == L.SEM_ERR_ARG and not h.value
    assert L.lib().sem_last_error()


def test_create_is_host_only_and_counts_unique_dof(L):
    rc, h = _create(L, 3, 32, 7)
    assert rc == L.SEM_OK
    assert L.lib().sem_ndof(h) == 3 * 224 ** 3
    L.lib().sem_destroy(h)
    # the largest 3D grid at N = 7 below 2^31 unknowns (E = 128 is refused above)
    rc, h = _create(L, 3, 127, 7)
    assert rc == L.SEM_OK
    assert L.lib().sem_ndof(h) == 3 * 889 ** 3 < 2 ** 31
    L.lib().sem_destroy(h)
    o = L.sem_opts(dim=3, E=2, N=15, nu=0.1, precision=L.SEM_PREC_FP32_BULK)
    h = ctypes.c_void_p()
    assert L.lib().sem_create_ex(ctypes.byref(o), ctypes.byref(h)) == L.SEM_OK
    L.lib().sem_destroy(h)
    o = L.sem_opts(dim=2, E=2, N=3, nu=0.1, ckpt_mode=L.SEM_CKPT_BINOMIAL, ckpt_slots=0)
    assert L.lib().sem_create_ex(ctypes.byref(o), ctypes.byref(h)) == L.SEM_ERR_ARG
    assert L.lib().sem_create(2, 2, 3, 0.1, None) == L.SEM_ERR_ARG


def test_null_handle_and_pointer_errors(L):
    assert L.lib().sem_rhs(None, None, None, None) == L.SEM_ERR_ARG
    rc, h = _create(L, 2, 3, 3)
    assert L.lib().sem_rhs(h, None, None, None) == L.SEM_ERR_ARG
    assert L.lib().sem_rk_adjoint(h, ctypes.c_void_p(64), ctypes.c_void_p(128), None) == L.SEM_ERR_STATE
    assert L.lib().sem_rhs(h, ctypes.c_void_p(8), ctypes.c_void_p(12), None) == L.SEM_ERR_ARG   # misaligned
    assert L.lib().sem_rhs(h, ctypes.c_void_p(4096), ctypes.c_void_p(4096 + 8), None) == L.SEM_ERR_ALIAS
    L.lib().sem_destroy(h)
    L.lib().sem_destroy(None)


@pytest.mark.parametrize("dim,E,N", [(1, 16, 7), (2, 5, 4), (3, 3, 15), (2, 1, 1)])
def test_host_gll_coordinates_match_oracle(L, dim, E, N):
    from paper_1806_01422_gb300 import Sem
    s = Sem(dim, E, N, 0.01, device="cpu")
    g = Grid(dim, E, N, 0.01)
    assert np.max(np.abs(s.coords() - g.coords())) < 1e-15 * g.L * 4
    assert s.ndof == g.ndof()


def test_checkpoint_planner_is_dp_optimal(L):
    from paper_1806_01422_gb300 import ckpt_plan
    for l in (1, 2, 3, 7, 12, 20, 30, 45):
        for s in range(0, 6):
            assert ckpt_plan(l, s) == optimal_advances(l, s), (l, s)
    # the binomial count for the 3D workload: 1000 steps, 20 slots (start + 19)
    assert ckpt_plan(1000, 19) == optimal_advances(1000, 19)
    with pytest.raises(Exception):
        ckpt_plan(0, 3)


def test_batch_create_validates_and_lays_out_packed_vectors(L):
    from paper_1806_01422_gb300 import SemBatch
    b = SemBatch([2, 3, 4], [5, 7, 9], [1e-3, 1e-3, 1e-3], device="cpu")
    offs = [o for o, _ in b.layout]
    sizes = [n for _, n in b.layout]
    assert sizes == [2 * (2 * 5) ** 2, 2 * (3 * 7) ** 2, 2 * (4 * 9) ** 2]
    assert offs == [0, sizes[0], sizes[0] + sizes[1]]
    assert b.ndof == sum(sizes)
    assert np.max(np.abs(b.coords(1) - Grid(2, 3, 7, 0.0).coords())) < 1e-15
    for bad in (([2], [4], [1e-3]), ([0], [5], [1e-3]), ([2], [5], [-1.0])):
        with pytest.raises(L.SemError):
            SemBatch(*bad, device="cpu")
    Ea = (ctypes.c_int * 1)(2)
    h = ctypes.c_void_p()
    assert L.lib().sem_batch_create(0, Ea, Ea, (ctypes.c_double * 1)(0.1), None, ctypes.byref(h)) == L.SEM_ERR_ARG
