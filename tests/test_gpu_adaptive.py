"""Adaptive step sizes (Sec. 5.1) on the GPU against the oracle's controller.

Both sides run the Bogacki-Shampine 3(2) pair with the same weighted RMS
error norm and controller in FP64.  Accept/reject decisions compare the norm
with 1, so the two sides take the same decisions unless a norm lies within
rounding of 1; the tests check that the accepted step sequences agree to
1e-12 relative, then compare states and gradients at 1e-10 relative (the step
sizes themselves carry the rounding differences of the norms).
"""
import numpy as np
import pytest
import torch

from oracle.sem import Grid
from oracle import adapt as oad
from oracle import rk as ork
from paper_1806_01422_gb300 import Sem, inputs
from paper_1806_01422_gb300 import _lib as L

pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1806_01422_gb300 import build
    build.build()


def relerr(got, ref):
    got = got.detach().cpu().numpy() if isinstance(got, torch.Tensor) else np.asarray(got)
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def test_fixed_step_bs3_matches_oracle():
    s, g = Sem(2, 3, 5, 0.02), Grid(2, 3, 5, 0.02)
    u0, uo = inputs.workload_field(2, g.coords(), 1), inputs.workload_field(2, g.coords(), 2)
    Jr, lam, uN = ork.objective_and_gradient(g, u0, uo, 2e-3, 10, "bs3")
    assert relerr(s.rk_forward(u0, 2e-3, 10, "bs3"), uN) < 1e-11
    J, grad = s.objective_grad(u0, uo, 2e-3, 10, "bs3")
    assert abs(J - Jr) <= 1e-11 * abs(Jr) and relerr(grad, lam) < 1e-11


@pytest.mark.parametrize("dim,E,N,nu,dt0,nsteps,tol", [(1, 8, 6, 0.02, 0.05, 10, 1e-6), (2, 3, 5, 0.01, 0.025, 2, 1e-7),
                                                     (3, 2, 4, 0.05, 1e-3, 20, 1e-8)])
def test_adaptive_sweep_matches_oracle(dim, E, N, nu, dt0, nsteps, tol):
    """sem_rk_forward(dt0, nsteps) runs over the horizon dt0 * nsteps from the trial step dt0."""
    s, g = Sem(dim, E, N, nu), Grid(dim, E, N, nu)
    x = g.coords()
    u0, uo = inputs.workload_field(dim, x, 1), inputs.workload_field(dim, x, 2)
    T = dt0 * nsteps
    uN, traj, dts, rej = oad.adaptive_forward(g.rhs, u0, T, dt0, tol, tol)
    J_ref, lamN = g.objective(uN, uo)
    lam0 = oad.adjoint_variable(g.jacT, traj, lamN, dts)
    s.set_adaptive(tol, tol)
    got = s.rk_forward(u0, dt0, nsteps, "bs3")
    gdts, grej = s.adaptive_steps()
    assert len(gdts) == len(dts) and grej == rej
    # each step size carries the rounding of all earlier error norms through err^(-1/3)
    assert np.max(np.abs(gdts - np.array(dts)) / np.array(dts)) < 1e-10
    assert abs(gdts.sum() - T) < 1e-13 * T
    assert relerr(got, uN) < RTOL
    J, grad = s.objective_grad(u0, uo, dt0, nsteps, "bs3")
    assert abs(J - J_ref) <= RTOL * abs(J_ref)
    assert relerr(grad, lam0) < RTOL
    assert s.trajectory_info()["device"] == len(dts) + 1


def test_adaptive_step_follows_a_stiffening_solution():
    """A sharpening Burgers front needs smaller steps later: the accepted steps are not uniform
    and the first trial step, far too large, is rejected."""
    s = Sem(1, 16, 6, 5e-3)
    x = s.coords()
    u0 = np.sin(x)[None, :]
    s.set_adaptive(1e-7, 1e-7)
    s.rk_forward(u0, 0.5, 2, "bs3")   # horizon 1.0, trial step 0.5
    dts, rej = s.adaptive_steps()
    assert rej >= 1 and dts.max() > 2 * dts.min()


def test_adaptive_argument_errors():
    s = Sem(2, 2, 4, 0.03, precision="fp32_bulk")
    with pytest.raises(L.SemError) as e:
        s.set_adaptive(1e-6, 1e-6)
    assert e.value.code == L.SEM_ERR_ARG
    s64 = Sem(2, 2, 4, 0.03)
    with pytest.raises(L.SemError) as e:
        s64.set_adaptive(-1.0, 0.0)
    assert e.value.code == L.SEM_ERR_ARG
