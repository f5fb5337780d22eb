"""GPU parity of the FP64-DF form (element kernels in double-float arithmetic).

Inputs, states, assembly and reductions are FP64; the contractions and pointwise
products run on pairs of floats with compensated dot products, rounding near
2^-48 relative to the magnitudes summed (about 32 times the FP64 unit
roundoff).  The results must meet the same 1e-11 relative bound as the FP64
form; the tests also record how close they come to the FP64 kernels.
"""
import numpy as np
import pytest
import torch

from oracle.sem import Grid
from oracle import rk as ork
from paper_1806_01422_gb300 import Sem, inputs

pytestmark = pytest.mark.gpu

RTOL64 = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1806_01422_gb300 import build
    build.build()


def relerr(got, ref):
    got = got.detach().cpu().numpy() if isinstance(got, torch.Tensor) else np.asarray(got)
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


OPS = [(1, 3, 3), (1, 16, 7), (1, 5, 15), (2, 1, 3), (2, 3, 4), (2, 5, 7), (2, 3, 15), (3, 1, 4), (3, 3, 7),
       (3, 2, 9), (3, 1, 10), (3, 2, 11), (3, 1, 15), (3, 2, 13)]


@pytest.mark.parametrize("dim,E,N", OPS)
def test_df_operators_match_oracle(dim, E, N):
    s, g = Sem(dim, E, N, 0.037, precision="fp64_df"), Grid(dim, E, N, 0.037)
    u, w = inputs.field_random(dim, g.G, 10 + N), inputs.field_random(dim, g.G, 20 + N)
    errs = {"F": relerr(s.rhs(u), g.rhs(u)), "J": relerr(s.jac(u, w), g.jac(u, w)),
            "JT": relerr(s.jacT(u, w), g.jacT(u, w))}
    assert max(errs.values()) < RTOL64, errs


@pytest.mark.parametrize("dim,E,N,scheme,steps,dt", [(2, 8, 7, "ssprk3", 20, 2e-4), (3, 3, 7, "rk4", 6, 2.5e-4),
                                                    (1, 16, 7, "rk4", 50, 1e-3)])
def test_df_gradient_matches_oracle(dim, E, N, scheme, steps, dt):
    nu = {1: 1e-2, 2: 1e-3, 3: 5e-4}[dim]
    s, g = Sem(dim, E, N, nu, precision="fp64_df"), Grid(dim, E, N, nu)
    x = g.coords()
    u0, uo = inputs.workload_field(dim, x, 1), inputs.workload_field(dim, x, 2)
    Jr, lam, uN = ork.objective_and_gradient(g, u0, uo, dt, steps, scheme)
    J, grad = s.objective_grad(u0, uo, dt, steps, scheme)
    assert abs(J - Jr) <= RTOL64 * abs(Jr)
    assert relerr(grad, lam) < RTOL64


def test_df_is_close_to_fp64_and_deterministic():
    dim, E, N = 2, 16, 7
    s, r = Sem(dim, E, N, 1e-3, precision="fp64_df"), Sem(dim, E, N, 1e-3)
    x = s.coords()
    u, w = inputs.workload_field(dim, x, 1), inputs.workload_field(dim, x, 2)
    a, b = s.jacT(u, w), r.jacT(u, w)
    err = float((a - b).abs().max() / b.abs().max())
    print("double-float vs FP64 J^T: %.2e" % err)
    assert err < 1e-12
    assert torch.equal(a, s.jacT(u, w))
