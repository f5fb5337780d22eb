"""Batched instances: packed results equal each instance's own handle bitwise,
and match the FP64 oracle; the autotuner picks one of its candidates."""
import numpy as np
import pytest
import torch

from oracle.sem import Grid
from oracle import rk as ork
from paper_1806_01422_gb300 import Sem, SemBatch, inputs

pytestmark = pytest.mark.gpu

E = [3, 5, 2, 4, 6, 1]
N = [5, 7, 9, 3, 7, 5]
NU = [1e-3, 2e-3, 1e-3, 5e-3, 1e-3, 1e-2]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1806_01422_gb300 import build
    build.build()


def fields(b, seed_base):
    return [inputs.field_2d(b.coords(k), seed_base + 2 * k) for k in range(b.count)]


def test_batched_operators_equal_each_instance_bitwise():
    b = SemBatch(E, N, NU)
    us, ws = fields(b, 1000), fields(b, 1001)
    u, w = torch.from_numpy(b.pack(us)).cuda(), torch.from_numpy(b.pack(ws)).cuda()
    F, Jw, JT = b.rhs(u).cpu().numpy(), b.jac(u, w).cpu().numpy(), b.jacT(u, w).cpu().numpy()
    for k in range(b.count):
        s = Sem(2, E[k], N[k], NU[k])
        for got, ref in ((F, s.rhs(us[k])), (Jw, s.jac(us[k], ws[k])), (JT, s.jacT(us[k], ws[k]))):
            assert np.array_equal(b.unpack(got)[k], ref.cpu().numpy()), k


@pytest.mark.parametrize("k", [1, 2, 5])
def test_batched_operators_match_oracle(k):
    b = SemBatch(E, N, NU)
    us, ws = fields(b, 1000), fields(b, 1001)
    u, w = torch.from_numpy(b.pack(us)).cuda(), torch.from_numpy(b.pack(ws)).cuda()
    g = Grid(2, E[k], N[k], NU[k])
    for got, ref in ((b.rhs(u), g.rhs(us[k])), (b.jacT(u, w), g.jacT(us[k], ws[k]))):
        x = b.unpack(got.cpu().numpy())[k]
        assert np.max(np.abs(x - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_batched_gradient_equals_each_instance_and_the_oracle():
    b = SemBatch(E, N, NU)
    u0s, uos = fields(b, 1000), fields(b, 1001)
    J, grad = b.objective_grad_each(b.pack(u0s), b.pack(uos), 1e-4, 12, "rk4")
    gk = b.unpack(grad.cpu().numpy())
    for k in range(b.count):
        s = Sem(2, E[k], N[k], NU[k])
        Jk, g1 = s.objective_grad(u0s[k], uos[k], 1e-4, 12, "rk4")
        assert np.array_equal(gk[k], g1.cpu().numpy()), k
        assert abs(J[k] - Jk) <= 1e-13 * abs(Jk)
    k = 1
    g = Grid(2, E[k], N[k], NU[k])
    Jr, lam, _ = ork.objective_and_gradient(g, u0s[k], uos[k], 1e-4, 12, "rk4")
    assert abs(J[k] - Jr) <= 1e-11 * abs(Jr)
    assert np.max(np.abs(gk[k] - lam)) <= 1e-11 * np.max(np.abs(lam))


def test_autotuner_picks_a_candidate_block_size():
    b = SemBatch(E, N, NU)
    threads, ms = b.autotune()
    assert threads in (64, 128, 192, 256)
    assert all(m > 0 for m in ms)
