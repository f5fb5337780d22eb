"""sem_rhs_noalloc: F(u) for callers that cannot allocate device memory.

Some callers of this library cannot call cudaMalloc when they need F(u): their
device memory belongs to their own pool or arena, or they run in loops that must
not take the device-wide synchronisation an allocation can cause.  The
allocation-free entry point keeps its only scratch in a fixed device array
inside libsem.so.  These tests call it through the C ABI:

* first, on a fresh handle that has never allocated its workspace, with the
  device's free memory read before and after the call (it must not change);
* then twice in a row, each result compared with sem_rhs on the same handle at
  the FP64 tolerance of the parity tests (1e-11 relative) and bitwise: the
  entry point runs the same element kernels (FP64, FP64-DF or FP32-bulk, as the
  handle's precision says) and the same gather-scatter as sem_rhs;
* a grid too large for the fixed array, and a batch handle, are refused.

The file name makes pytest collect it last.
"""
import ctypes

import pytest
import torch

from paper_1806_01422_gb300 import Sem, SemBatch, inputs
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


CASES = [(2, 64, 7, "fp64"), (3, 6, 7, "fp64"), (1, 16, 7, "fp64"), (3, 8, 7, "fp32_bulk"),
         (2, 16, 7, "fp64_df"), (3, 5, 5, "fp64_df")]


@pytest.mark.parametrize("dim,E,N,prec", CASES)
def test_allocation_free_rhs_matches_sem_rhs_on_two_calls(dim, E, N, prec):
    # load the kernels (lazy module loading allocates on the first launch) on a throwaway handle
    warm = Sem(dim, E, N, 1e-3, precision=prec)
    x = warm.coords()
    u = torch.from_numpy(inputs.workload_field(dim, x, inputs.SEED_U0)).cuda()
    out = torch.full_like(u, float("nan"))
    assert _noalloc(warm, u, out) == L.SEM_OK, L.lib().sem_last_error()
    torch.cuda.synchronize()
    warm.close()

    # a fresh handle: the entry point runs before the handle has any workspace
    s = Sem(dim, E, N, 1e-3, precision=prec)
    outs = [torch.full_like(u, float("nan")) for _ in range(2)]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for o in outs:
        assert _noalloc(s, u, o) == L.SEM_OK, L.lib().sem_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)

    ref = s.rhs(u).clone()
    for o in outs:
        err = float((o - ref).abs().max() / ref.abs().max())
        assert err <= RTOL64, err
        assert torch.equal(o, ref)   # the same kernels on the same inputs as sem_rhs
    s.close()


def test_allocation_free_rhs_refuses_grids_beyond_its_scratch():
    s = Sem(3, 32, 7, 1e-3)      # needs 3 * 32^3 * 8^3 doubles, far above the fixed array
    u = torch.zeros(s.shape, dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    assert _noalloc(s, u, out) == L.SEM_ERR_ARG
    assert b"scratch" in L.lib().sem_last_error()


def test_allocation_free_rhs_refuses_batch_handles():
    b = SemBatch([4, 8], [5, 7], [1e-3, 1e-3])
    u = torch.zeros(b.ndof, dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    assert _noalloc(b, u, out) == L.SEM_ERR_ARG
    assert b"batch" in L.lib().sem_last_error()
