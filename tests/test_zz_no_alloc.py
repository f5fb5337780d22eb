"""sem_rhs_noalloc: F(u) for callers that cannot allocate device memory.

Some callers of this library cannot call cudaMalloc when they need F(u) (their
device memory belongs to their own pool, or they run in loops that must not
take the synchronisation an allocation can cause).  The allocation-free entry
point keeps its scratch in a fixed device array inside libsem.so.  This test
calls it through the C ABI twice in a row and compares each result with
sem_rhs on the same handle, at the FP64 tolerance of the parity tests; it also
checks that a grid too large for the fixed array is refused.  The file name
makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1806_01422_gb300 import Sem, inputs
from paper_1806_01422_gb300 import _lib as L

pytestmark = pytest.mark.gpu

RTOL64 = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1806_01422_gb300 import build
    build.build()


def _noalloc(s, u, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.lib().sem_rhs_noalloc(s._h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(out.data_ptr()), stream)


@pytest.mark.parametrize("dim,E,N,prec", [(2, 64, 7, "fp64"), (3, 6, 7, "fp64"), (1, 16, 7, "fp64"),
                                          (3, 8, 7, "fp32_bulk")])
def test_allocation_free_rhs_matches_sem_rhs_on_two_calls(dim, E, N, prec):
    s = Sem(dim, E, N, 1e-3, precision=prec)
    x = s.coords()
    u = torch.from_numpy(inputs.workload_field(dim, x, inputs.SEED_U0)).cuda()
    ref = s.rhs(u).clone()
    for _ in range(2):
        out = torch.full_like(u, float("nan"))
        assert _noalloc(s, u, out) == L.SEM_OK, L.lib().sem_last_error()
        torch.cuda.synchronize()
        err = float((out - ref).abs().max() / ref.abs().max())
        assert err <= RTOL64, err


def test_allocation_free_rhs_refuses_grids_beyond_its_scratch():
    s = Sem(3, 32, 7, 1e-3)      # needs 3 * 32^3 * 8^3 doubles, far above the fixed array
    u = torch.zeros(s.shape, dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    assert _noalloc(s, u, out) == L.SEM_ERR_ARG
    assert b"scratch" in L.lib().sem_last_error()
