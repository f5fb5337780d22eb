"""Workloads with exact solutions (Sec. 6.1) on the GPU.

* Frozen advection (du/dt = J(a) u): the library's sweeps against the oracle's
  sweeps with F = J(a) . and J^T = J(a)^T . (FP64, 1e-11 relative), for every
  RK scheme and for Crank-Nicolson.
* The advection-diffusion inverse problem of the paper's convergence study
  (nu = 1e-5, a = 0.1, T = 0.01, five modes): L-BFGS over library gradients
  recovers the initial condition; its error against the exact initial
  condition falls at a rate of at least 2 under h-refinement and faster than
  geometrically under p-refinement.
* The Cole-Hopf inverse problem (Sec. 6.1.1): from the exact initial condition
  plus a Gaussian, L-BFGS drives the misfit down by more than 1e6 and the
  initial-condition error down by a factor of 3 (the Gaussian's high modes are
  damped out of the observation, so the error stagnates, as the paper notes).
"""
import math

import numpy as np
import pytest
import torch

from oracle.sem import Grid
from oracle import rk as ork
from oracle import cn as ocn
from paper_1806_01422_gb300 import Sem, inputs
from paper_1806_01422_gb300.inverse import recover_initial_condition

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1806_01422_gb300 import build
    build.build()


def relerr(got, ref):
    got = got.detach().cpu().numpy() if isinstance(got, torch.Tensor) else np.asarray(got)
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


@pytest.mark.parametrize("dim,E,N,scheme,ckpt", [(1, 6, 7, "rk4", "auto"), (2, 3, 5, "ssprk3", "stages"),
                                                 (3, 2, 4, "rk4", "binomial"), (2, 3, 4, "euler", "states")])
def test_frozen_advection_sweeps_match_oracle(dim, E, N, scheme, ckpt):
    nu, dt, steps = 0.02, 2e-3, 12
    s, g = Sem(dim, E, N, nu, ckpt=ckpt, ckpt_slots=3), Grid(dim, E, N, nu)
    x = g.coords()
    a = inputs.workload_field(dim, x, 5)          # a non-constant field: the -(u.grad) a term is active
    u0, uo = inputs.workload_field(dim, x, 1), inputs.workload_field(dim, x, 2)
    F = lambda u: g.jac(a, u)
    JT = lambda Y, v: g.jacT(a, v)
    uN, traj = ork.rk_forward(F, u0, dt, steps, scheme)
    Jr, lamN = g.objective(uN, uo)
    lam0 = ork.rk_adjoint(JT, traj, lamN, dt, scheme)
    s.set_advection(a)
    assert relerr(s.rk_forward(u0, dt, steps, scheme), uN) < 1e-11
    J, grad = s.objective_grad(u0, uo, dt, steps, scheme)
    assert abs(J - Jr) <= 1e-11 * abs(Jr)
    assert relerr(grad, lam0) < 1e-11
    # back to Burgers
    s.set_advection(None)
    Jb, lb, _ = ork.objective_and_gradient(g, u0, uo, dt, steps, scheme)
    J2, g2 = s.objective_grad(u0, uo, dt, steps, scheme)
    assert abs(J2 - Jb) <= 1e-11 * abs(Jb) and relerr(g2, lb) < 1e-11


def test_frozen_advection_with_crank_nicolson_matches_oracle():
    dim, E, N, nu, dt, steps = 2, 2, 4, 0.03, 0.02, 3
    s, g = Sem(dim, E, N, nu), Grid(dim, E, N, nu)
    x = g.coords()
    a = inputs.workload_field(dim, x, 5)
    u0, uo = inputs.workload_field(dim, x, 1), inputs.workload_field(dim, x, 2)
    jac_a = lambda u, w: g.jac(a, w)
    uN, traj = ocn.cn_forward(lambda u: g.jac(a, u), jac_a, u0, dt, steps)
    Jr, lamN = g.objective(uN, uo)
    Aden = ocn.assembled_jacobian(jac_a, u0)
    lam0 = ocn.cn_adjoint(lambda u: Aden.T, traj, lamN, dt)
    s.set_advection(a)
    J, grad = s.objective_grad(u0, uo, dt, steps, "cn")
    assert abs(J - Jr) <= 1e-9 * abs(Jr)
    assert relerr(grad, lam0) < 1e-9
    assert s.solver_stats()["newton"] <= 2 * steps     # a linear step converges in one or two iterations


def _advection_diffusion_error(E, N):
    nu, a, T = 1e-5, 0.1, 0.01
    s = Sem(1, E, N, nu, L_box=1.0)
    x = s.coords()
    c_true, c_guess = inputs.advection_diffusion_coefs(5), inputs.advection_diffusion_coefs(6)
    s.set_advection(np.full((1, s.G), a))
    steps = 100
    dt = T / steps
    u_obs = inputs.advection_diffusion_1d(x, T, c_true, nu, a)
    u_true = torch.from_numpy(inputs.advection_diffusion_1d(x, 0.0, c_true, nu, a)).cuda()
    u_init = inputs.advection_diffusion_1d(x, 0.0, c_guess, nu, a)
    est, hist = recover_initial_condition(s, u_obs, u_init, dt, steps, "rk4", iters=60)
    assert hist[-1][1] < 1e-20 * hist[0][1] + 1e-28
    # L2 error through the GLL mass: sqrt(2 J(est; u_true)) with the misfit of the handle
    return math.sqrt(2.0 * s.objective(est, u_true))


def test_advection_diffusion_inverse_problem_h_refinement():
    errs = [_advection_diffusion_error(E, 3) for E in (8, 16, 32)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 2.0, (errs, rates)


def test_advection_diffusion_inverse_problem_p_refinement():
    errs = [_advection_diffusion_error(4, N) for N in (4, 6, 8)]
    # spectral: each +2 in the order gains more than the previous step did
    assert errs[1] < errs[0] / 5 and errs[2] < errs[1] / 10, errs


def test_cole_hopf_inverse_problem_from_a_perturbed_guess():
    nu, T = 0.05, 4.0
    s = Sem(1, 8, 6, nu, L_box=4.0)
    x = s.coords()
    steps = 800
    u_obs = inputs.cole_hopf_1d(x, T, nu)
    u_true = torch.from_numpy(inputs.cole_hopf_1d(x, 0.0, nu)).cuda()
    u_init = inputs.cole_hopf_1d(x, 0.0, nu) + inputs.gaussian_bump(x)
    est, hist = recover_initial_condition(s, u_obs, u_init, T / steps, steps, "rk4", iters=60)
    assert hist[-1][1] < 1e-6 * hist[0][1]
    assert all(b[1] <= a[1] for a, b in zip(hist, hist[1:]))
    err0 = math.sqrt(2.0 * s.objective(torch.from_numpy(u_init).cuda(), u_true))
    errn = math.sqrt(2.0 * s.objective(est, u_true))
    assert errn < err0 / 3
