"""GPU parity of the Crank-Nicolson scheme (Sec. 6.3) against the dense FP64 oracle.

The library solves each Newton system and each adjoint system with restarted
GMRES to a relative residual of 1e-12 and stops Newton at a relative step of
1e-12; the oracle solves them directly.  Both errors stay near 1e-12 per step,
so states, misfits and gradients over a few steps agree to 1e-9 relative.
"""
import numpy as np
import pytest
import torch

from oracle.sem import Grid
from oracle import cn as ocn
from paper_1806_01422_gb300 import Sem, inputs
from paper_1806_01422_gb300 import _lib as L

pytestmark = pytest.mark.gpu

RTOL_CN = 1e-9

# (dim, E, N, nu, dt, steps): dt is far above the explicit limit in the last two
CASES = [(1, 6, 5, 0.02, 0.05, 6), (2, 2, 4, 0.03, 0.01, 4), (3, 1, 3, 0.05, 0.02, 3), (2, 3, 5, 0.2, 0.05, 3)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1806_01422_gb300 import build
    build.build()


def relerr(got, ref):
    got = got.detach().cpu().numpy() if isinstance(got, torch.Tensor) else np.asarray(got)
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def fields(g):
    return inputs.workload_field(g.d, g.coords(), 1), inputs.workload_field(g.d, g.coords(), 2)


@pytest.mark.parametrize("dim,E,N,nu,dt,steps", CASES)
def test_cn_forward_matches_oracle(dim, E, N, nu, dt, steps):
    s, g = Sem(dim, E, N, nu), Grid(dim, E, N, nu)
    u0, _ = fields(g)
    ref, _ = ocn.cn_forward(g.rhs, g.jac, u0, dt, steps)
    got = s.rk_forward(u0, dt, steps, "cn")
    assert relerr(got, ref) < RTOL_CN
    st = s.solver_stats()
    assert st["newton"] >= steps and st["forward_krylov"] > 0


@pytest.mark.parametrize("dim,E,N,nu,dt,steps", CASES)
def test_cn_gradient_matches_oracle(dim, E, N, nu, dt, steps):
    s, g = Sem(dim, E, N, nu), Grid(dim, E, N, nu)
    u0, uo = fields(g)
    Jr, lam_ref, _ = ocn.cn_objective_and_gradient(g, u0, uo, dt, steps)
    J, grad = s.objective_grad(u0, uo, dt, steps, "cn")
    assert abs(J - Jr) <= RTOL_CN * abs(Jr)
    assert relerr(grad, lam_ref) < RTOL_CN
    assert s.solver_stats()["adjoint_krylov"] > 0


def test_cn_restarted_gmres_gives_the_same_gradient():
    dim, E, N, nu, dt, steps = CASES[1]
    s, g = Sem(dim, E, N, nu), Grid(dim, E, N, nu)
    u0, uo = fields(g)
    Jr, lam_ref, _ = ocn.cn_objective_and_gradient(g, u0, uo, dt, steps)
    s.set_solver(krylov_m=3)     # forces many restarts
    J, grad = s.objective_grad(u0, uo, dt, steps, "cn")
    assert abs(J - Jr) <= RTOL_CN * abs(Jr)
    assert relerr(grad, lam_ref) < RTOL_CN


def test_cn_adjoint_sweep_is_the_transpose_of_the_tangent():
    dim, E, N, nu, dt, steps = CASES[1]
    s, g = Sem(dim, E, N, nu), Grid(dim, E, N, nu)
    u0, _ = fields(g)
    _, traj = ocn.cn_forward(g.rhs, g.jac, u0, dt, steps)
    rng = np.random.default_rng(7)
    du0, lamT = rng.standard_normal(u0.shape), rng.standard_normal(u0.shape)
    duN = ocn.cn_tangent(lambda u: ocn.assembled_jacobian(g.jac, u), traj, du0, dt)
    s.rk_forward(u0, dt, steps, "cn")
    lam0 = s.rk_adjoint(lamT).cpu().numpy()
    lhs, rhs = float(np.sum(lamT * duN)), float(np.sum(lam0 * du0))
    assert abs(lhs - rhs) <= 1e-9 * max(abs(lhs), 1.0)


def test_cn_with_graph_enabled_runs_without_capture():
    dim, E, N, nu, dt, steps = CASES[0]
    s, g = Sem(dim, E, N, nu), Grid(dim, E, N, nu)
    u0, uo = fields(g)
    J0, g0 = s.objective_grad(u0, uo, dt, steps, "cn")
    s.use_graph(True)
    J1, g1 = s.objective_grad(u0, uo, dt, steps, "cn")
    assert s.graph_replays() == 0
    assert J0 == J1 and torch.equal(g0, g1)


def test_cn_argument_errors():
    s = Sem(2, 2, 4, 0.03, precision="fp32_bulk")
    with pytest.raises(L.SemError) as e:
        s.rk_forward(np.zeros(s.shape), 0.01, 2, "cn")
    assert e.value.code == L.SEM_ERR_ARG
    s64 = Sem(2, 2, 4, 0.03)
    for bad in [dict(newton_rtol=0.0), dict(krylov_m=0), dict(krylov_m=39), dict(krylov_maxit=0)]:
        with pytest.raises(L.SemError) as e:
            s64.set_solver(**bad)
        assert e.value.code == L.SEM_ERR_ARG
    s64.set_solver(krylov_rtol=1e-12, krylov_maxit=1)   # one Arnoldi step cannot reach 1e-12
    with pytest.raises(L.SemError) as e:
        s64.rk_forward(inputs.field_random(2, 8, 3), 0.01, 1, "cn")
    assert e.value.code == L.SEM_ERR_NONFINITE
