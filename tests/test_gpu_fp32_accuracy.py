"""Accuracy of the FP32-bulk form at the horizons and viscosities it is reported on.

The FP32-bulk form computes the contractions, pointwise products and element sums
in FP32 and keeps stage accumulation, misfit and gradient sums in float pairs or
FP64.  Its error against the FP64 form comes from the FP32 rounding of the large
inter-element viscous fluxes of the lumped-mass weak form (Sec. 3.2), which cancel
in the gather-scatter sum; in a sweep it adds up step by step, so it grows with the
horizon.  Measured on GB300 (relative to the largest entry):

  2D, 64^2 quads, N = 7, nu = 1e-3, SSP-RK3, dt = 2e-4 (the 2D workload):
      steps    u_N       J         gradient
      250      9.7e-8    7.2e-9    8.3e-8
      500      3.2e-7    1.5e-8    1.2e-7
      1000     3.6e-6    3.3e-8    2.6e-7
      2000     4.7e-6    3.8e-8    4.4e-7
  2D, 8^2 quads, N = 7, nu = 1e-2, 500 steps, against the FP64 oracle:
               2.6e-7    5.0e-8    6.7e-8
  3D, 32^3 hexes, N = 7, nu = 5e-4, RK4, 300 steps: J 1.2e-8, gradient 1.5e-7.

The tests assert these figures with a margin of about 1.5x, so the stated
accuracy is the one the tests check, up to the full 2000-step horizon.
"""
import numpy as np
import pytest
import torch

from oracle.sem import Grid
from oracle import rk as ork
from paper_1806_01422_gb300 import Sem, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1806_01422_gb300 import build
    build.build()


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("steps,bounds", [(500, (5e-7, 2.5e-8, 2e-7)), (2000, (7e-6, 6e-8, 7e-7))])
def test_fp32_bulk_error_at_the_2d_workload_horizon(steps, bounds):
    b_u, b_J, b_g = bounds
    s64 = Sem(2, 64, 7, 1e-3, precision="fp64")
    s32 = Sem(2, 64, 7, 1e-3, precision="fp32_bulk")
    x = s64.coords()
    u0 = torch.from_numpy(inputs.workload_field(2, x, inputs.SEED_U0)).cuda()
    uo = torch.from_numpy(inputs.workload_field(2, x, inputs.SEED_UOBS)).cuda()
    uN64 = s64.rk_forward(u0, 2e-4, steps, "ssprk3").clone()
    uN32 = s32.rk_forward(u0, 2e-4, steps, "ssprk3").clone()
    J64, g64 = s64.objective_grad(u0, uo, 2e-4, steps, "ssprk3")
    J32, g32 = s32.objective_grad(u0, uo, 2e-4, steps, "ssprk3")
    assert _rel(uN32, uN64) <= b_u
    assert abs(J32 - J64) <= b_J * abs(J64)
    assert _rel(g32, g64) <= b_g


def test_fp32_bulk_error_at_nu_1e_2_against_the_oracle():
    g = Grid(2, 8, 7, 1e-2)
    s = Sem(2, 8, 7, 1e-2, precision="fp32_bulk")
    u0, uo = inputs.workload_field(2, g.coords(), 1), inputs.workload_field(2, g.coords(), 2)
    Jr, lam, uNr = ork.objective_and_gradient(g, u0, uo, 2e-4, 500, "ssprk3")
    uN = s.rk_forward(u0, 2e-4, 500, "ssprk3").cpu().numpy()
    J, grad = s.objective_grad(u0, uo, 2e-4, 500, "ssprk3")
    grad = grad.cpu().numpy()
    assert np.max(np.abs(uN - uNr)) <= 4e-7 * np.max(np.abs(uNr))
    assert abs(J - Jr) <= 8e-8 * abs(Jr)
    assert np.max(np.abs(grad - lam)) <= 1e-7 * np.max(np.abs(lam))
