"""Pins of the FP64 CPU oracle against the mathematics (no GPU).

Each test checks the oracle against something other than itself: exact GLL
quadrature, exact polynomial derivatives, closed-form PDE solutions, exact
central differences of a quadratic map, transposes of assembled Jacobians,
Taylor polynomials of exp(dt A), brute-force schedules and the paper's printed
unknown counts.
"""
import os
from math import comb

import numpy as np
import pytest

from oracle.gll import gll
from oracle.sem import Grid
from oracle import rk as ork
from oracle.checkpoint import optimal_advances, checkpointed_gradient_lam0
from oracle import adapt as oad
from paper_1806_01422_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- GLL (Sec. 3.2)
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7, 9, 15])
def test_gll_nodes_are_legendre_lobatto_points(N):
    x, w, D = gll(N)
    assert x[0] == -1.0 and x[-1] == 1.0
    if N > 1:
        roots = np.sort(np.polynomial.legendre.Legendre.basis(N).deriv().roots().real)
        assert np.max(np.abs(roots - x[1:-1])) < 1e-14


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7, 9, 15])
def test_gll_quadrature_exact_to_degree_2N_minus_1(N):
    x, w, D = gll(N)
    for k in range(2 * N):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14 * max(1.0, 2 ** k)
    # degree 2N is NOT integrated exactly (GLL has precision 2N-1)
    assert abs(np.dot(w, x ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-12


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7, 9, 15])
def test_derivative_matrix_exact_on_polynomials(N):
    x, w, D = gll(N)
    rng = np.random.default_rng(N)
    p = np.polynomial.Polynomial(rng.standard_normal(N + 1))
    assert np.max(np.abs(D @ p(x) - p.deriv()(x))) < 1e-11 * (N + 1) ** 2
    assert np.max(np.abs(D @ np.ones(N + 1))) < 1e-12 * (N + 1) ** 2
    # centro-antisymmetry D[n-1-i, n-1-j] = -D[i, j] (symmetric node set)
    assert np.max(np.abs(D[::-1, ::-1] + D)) < 1e-12 * (N + 1) ** 2


@pytest.mark.parametrize("N", [2, 3, 5, 7, 15])
def test_stiffness_is_exact_energy(N):
    """K = D^T W D gives u^T K u = int (u')^2 exactly for degree <= N (Sec. 3.2, K = D^T M D)."""
    x, w, D = gll(N)
    K = D.T @ np.diag(w) @ D
    rng = np.random.default_rng(10 + N)
    p = np.polynomial.Polynomial(rng.standard_normal(N + 1))
    dp2 = p.deriv() ** 2
    exact = dp2.integ()(1.0) - dp2.integ()(-1.0)
    u = p(x)
    assert abs(u @ K @ u - exact) < 1e-10 * max(1.0, abs(exact))
    assert np.max(np.abs(K - K.T)) < 1e-12 * np.max(np.abs(K))
    ev = np.linalg.eigvalsh(K)
    assert ev[0] > -1e-10 * ev[-1] and np.sum(np.abs(ev) < 1e-9 * ev[-1]) == 1


# ------------------------------------------------------ layout and unknown counts
def test_unique_dof_count_matches_paper():
    path = os.path.join(HERE, "golden", "paper_dof_counts.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 4
    for E, pts, printed, *_ in rows[:3]:
        N = int(pts) - 1
        assert 3 * (int(E) * N) ** 3 == int(printed)
    E, pts, printed = int(rows[3][0]), int(rows[3][1]), int(rows[3][2])
    assert E * 3 * (pts - 1) ** 3 == printed
    assert Grid(3, 2, 3, 0.0).ndof() == 3 * 6 ** 3


def test_mass_is_gll_quadrature_of_the_box():
    for dim, E, N in [(1, 4, 8), (2, 3, 7), (3, 2, 9)]:
        g = Grid(dim, E, N, 0.0)
        assert abs(g.M.sum() - g.L ** dim) < 1e-12 * g.L ** dim
        # integrates a smooth periodic function spectrally: int sin^2(2 pi x / L) = L^d / 2
        x = g.coords()
        f = np.sin(2 * np.pi * x / g.L) ** 2
        shape = [1] * dim
        shape[-1] = x.size
        F = np.broadcast_to(f.reshape(shape), g.global_shape())
        assert abs((g.M * F).sum() - g.L ** dim / 2) < 1e-6 * g.L ** dim


def test_gather_scatter_are_transposes():
    g = Grid(3, 3, 2, 0.0)
    rng = np.random.default_rng(0)
    u = rng.standard_normal(g.global_shape())
    U = rng.standard_normal(g.local_shape())
    assert abs(np.sum(g.gather(u) * U) - np.sum(u * g.scatter_add(U))) < 1e-12 * np.abs(U).sum()
    counts = g.scatter_add(np.ones(g.local_shape()))
    assert set(np.unique(counts)) == {1.0, 2.0, 4.0, 8.0}


# --------------------------------------------------- the operator F (eq. rhsvec)
@pytest.mark.parametrize("dim", [1, 2, 3])
def test_rhs_of_constant_field_is_zero(dim):
    g = Grid(dim, 3, 4, 0.1)
    u = np.stack([np.full(g.global_shape(), 0.7 - 0.3 * c) for c in range(dim)])
    assert np.max(np.abs(g.rhs(u))) < 1e-12


def _mesh(g):
    x = g.coords()
    return np.meshgrid(*([x] * g.d), indexing="ij")[::-1] if g.d > 1 else [x]


def test_rhs_1d_converges_to_burgers_terms():
    """Viscous part -> nu u_xx and advective part -> -u u_x spectrally (Eq. burgers23d)."""
    for k in (1, 3):
        g0, g1 = Grid(1, 16, 9, 0.0), Grid(1, 16, 9, 1.0)
        x = g0.coords()
        u = np.sin(k * x)[None]
        visc = g1.rhs(u) - g0.rhs(u)
        assert np.max(np.abs(visc[0] + k * k * np.sin(k * x))) < 1e-7 * k * k
        adv = g0.rhs(u)
        assert np.max(np.abs(adv[0] + k * np.sin(k * x) * np.cos(k * x))) < 1e-7 * k


def test_rhs_2d_and_3d_converge_to_burgers_operator():
    nu = 0.01
    # 2D: u = (sin 2pi x cos 2pi y, 0.5 cos 2pi x sin 4pi y); X = x_0 along last axis
    g = Grid(2, 8, 9, nu)
    X, Y = _mesh(g)
    tp = 2 * np.pi
    ux, uy = np.sin(tp * X) * np.cos(tp * Y), 0.5 * np.cos(tp * X) * np.sin(2 * tp * Y)
    dux = (tp * np.cos(tp * X) * np.cos(tp * Y), -tp * np.sin(tp * X) * np.sin(tp * Y))
    duy = (-0.5 * tp * np.sin(tp * X) * np.sin(2 * tp * Y), tp * np.cos(tp * X) * np.cos(2 * tp * Y))
    lapx, lapy = -2 * tp * tp * ux, -5 * tp * tp * uy
    F = g.rhs(np.stack([ux, uy]))
    ex = nu * lapx - (ux * dux[0] + uy * dux[1])
    ey = nu * lapy - (ux * duy[0] + uy * duy[1])
    assert np.max(np.abs(F[0] - ex)) < 1e-6 and np.max(np.abs(F[1] - ey)) < 1e-6
    # 3D: the paper's initial condition (Sec. 6.2), period 4 in every direction
    g = Grid(3, 4, 9, nu, L=4.0)
    X, Y, Z = _mesh(g)
    hp = 0.5 * np.pi
    s, c = np.sin, np.cos
    u = [s(hp * X) * c(hp * Y) * c(hp * Z), s(hp * Y) * c(hp * Z) * c(hp * X), s(hp * Z) * c(hp * X) * c(hp * Y)]
    F = g.rhs(np.stack(u))
    # u_1 = s(X)c(Y)c(Z) etc.; grad and Laplacian in closed form (Lap = -3 hp^2 u)
    grads = [
        (hp * c(hp * X) * c(hp * Y) * c(hp * Z), -hp * s(hp * X) * s(hp * Y) * c(hp * Z), -hp * s(hp * X) * c(hp * Y) * s(hp * Z)),
        (-hp * s(hp * Y) * c(hp * Z) * s(hp * X), hp * c(hp * Y) * c(hp * Z) * c(hp * X), -hp * s(hp * Y) * s(hp * Z) * c(hp * X)),
        (-hp * s(hp * Z) * s(hp * X) * c(hp * Y), -hp * s(hp * Z) * c(hp * X) * s(hp * Y), hp * c(hp * Z) * c(hp * X) * c(hp * Y)),
    ]
    for comp in range(3):
        exact = nu * (-3 * hp * hp) * u[comp] - sum(u[j] * grads[comp][j] for j in range(3))
        assert np.max(np.abs(F[comp] - exact)) < 1e-6


# ----------------------------------------- J (eq. jacvec) and J^T (eq. jactransvec)
SMALL = [(1, 3, 3), (1, 4, 5), (2, 2, 3), (2, 3, 2), (3, 2, 2), (3, 2, 3)]


@pytest.mark.parametrize("dim,E,N", SMALL)
def test_jacobian_is_exact_central_difference(dim, E, N):
    """F is quadratic in u, so (F(u+ew) - F(u-ew)) / 2e equals J(u)w up to roundoff for any e."""
    g = Grid(dim, E, N, 0.037)
    rng = np.random.default_rng(dim * 100 + E * 10 + N)
    u, w = rng.standard_normal((2, dim) + g.global_shape())
    Jw = g.jac(u, w)
    for eps in (1.0, 1e-2):
        fd = (g.rhs(u + eps * w) - g.rhs(u - eps * w)) / (2 * eps)
        assert np.max(np.abs(fd - Jw)) < 1e-11 * np.max(np.abs(Jw)) / min(eps, 1.0)


def _assembled_jacobian(g, u):
    """Dense Jacobian from exact central differences of F, column by column (Sec. 6 check)."""
    n = g.ndof()
    cols = []
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        e = e.reshape(u.shape)
        cols.append(((g.rhs(u + e) - g.rhs(u - e)) / 2.0).ravel())
    return np.array(cols).T


@pytest.mark.parametrize("dim,E,N", SMALL)
def test_transpose_matches_assembled_jacobian_entry_by_entry(dim, E, N):
    """The paper's check: explicit J from the identity, its transpose vs the matrix-free J^T."""
    g = Grid(dim, E, N, 0.05)
    rng = np.random.default_rng(7 + dim)
    u = rng.standard_normal((dim,) + g.global_shape())
    Jd = _assembled_jacobian(g, u)
    n = g.ndof()
    JT_cols = np.array([g.jacT(u, np.eye(n)[k].reshape(u.shape)).ravel() for k in range(n)]).T
    assert np.max(np.abs(JT_cols - Jd.T)) < 1e-11 * np.max(np.abs(Jd))


@pytest.mark.parametrize("dim,E,N", [(1, 16, 7), (2, 4, 7), (3, 3, 7)])
def test_dot_product_identity(dim, E, N):
    g = Grid(dim, E, N, 0.01)
    rng = np.random.default_rng(3)
    u, w, v = rng.standard_normal((3, dim) + g.global_shape())
    Jw = g.jac(u, w)
    lhs, rhs = np.sum(Jw * v), np.sum(w * g.jacT(u, v))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Jw) * np.linalg.norm(v)


def test_transpose_of_viscous_part_is_mass_similar():
    """With u = 0 only the viscous term is left: J^T = M J M^-1 (K symmetric, Sec. 3.3)."""
    g = Grid(2, 3, 4, 0.3)
    rng = np.random.default_rng(5)
    u = np.zeros((2,) + g.global_shape())
    v = rng.standard_normal(u.shape)
    assert np.max(np.abs(g.jacT(u, v) - g.M * g.jac(u, v / g.M))) < 1e-12 * np.max(np.abs(g.jacT(u, v)))


# ------------------------------------------------------- objective (eq. ourcost)
def test_objective_closed_forms():
    g = Grid(3, 2, 3, 0.0)
    u = np.full((3,) + g.global_shape(), 0.25)
    J, lam = g.objective(u, np.zeros_like(u))
    assert abs(J - 0.5 * 0.25 ** 2 * 3 * g.L ** 3) < 1e-14
    rng = np.random.default_rng(1)
    u, uo, du = rng.standard_normal((3, 3) + g.global_shape())
    J0, lam = g.objective(u, uo)
    eps = 1e-4
    fd = (g.objective(u + eps * du, uo)[0] - g.objective(u - eps * du, uo)[0]) / (2 * eps)
    assert abs(fd - np.sum(lam * du)) < 1e-9 * abs(fd)


# ----------------------------------------------------- RK sweeps (Sec. 4.1)
@pytest.mark.parametrize("scheme,order", [("rk4", 4), ("ssprk3", 3), ("euler", 1), ("bs3", 3)])
def test_rk_step_is_taylor_polynomial_on_linear_problems(scheme, order):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((6, 6))
    dt = 0.3
    u = rng.standard_normal(6)
    un, _ = ork.rk_step(lambda y: A @ y, u, dt, scheme)
    P = sum(np.linalg.matrix_power(dt * A, k) / np.prod(range(1, k + 1)) for k in range(order + 1))
    assert np.max(np.abs(un - P @ u)) < 1e-13 * np.max(np.abs(P @ u))
    lam = rng.standard_normal(6)
    back = ork.rk_adjoint_step(lambda y, v: A.T @ v, [None] * len(ork.TABLEAUX[scheme][1]), lam, dt, scheme)
    assert np.max(np.abs(back - P.T @ lam)) < 1e-13 * np.max(np.abs(P.T @ lam))


def test_forward_euler_adjoint_is_the_papers_recursion():
    """Sec. 4.1: for forward Euler v_n = v_{n+1} + dt J^T v_{n+1}."""
    g = Grid(2, 2, 3, 0.02)
    rng = np.random.default_rng(8)
    u, lam = rng.standard_normal((2, 2) + g.global_shape())
    _, Y = ork.rk_step(g.rhs, u, 1e-3, "euler")
    got = ork.rk_adjoint_step(g.jacT, Y, lam, 1e-3, "euler")
    assert np.max(np.abs(got - (lam + 1e-3 * g.jacT(u, lam)))) < 1e-15 * np.max(np.abs(lam)) * 10


def test_cole_hopf_solution_is_reproduced():
    """Sec. 6.1.1 exact 1D viscous Burgers solution, periodic with period 2 (box [0, 4))."""
    nu = 0.05

    def exact(x, t):
        e = np.exp(-nu * t * np.pi ** 2)
        return 2 * nu * np.pi * np.sin(np.pi * x) * e / (2 + e * np.cos(np.pi * x))

    g = Grid(1, 16, 9, nu, L=4.0)
    x = g.coords()
    T, steps = 0.5, 1000   # dt inside the explicit viscous stability limit
    uT, _ = ork.rk_forward(g.rhs, exact(x, 0.0)[None], T / steps, steps, "rk4")
    assert np.max(np.abs(uT[0] - exact(x, T))) < 1e-9
    # the sign of either term flipped would be visible at this level
    assert np.max(np.abs(exact(x, T) - exact(x, 0.0))) > 1e-3


@pytest.mark.parametrize("dim,scheme", [(1, "rk4"), (2, "ssprk3"), (3, "rk4")])
def test_tangent_adjoint_duality_over_trajectory(dim, scheme):
    g = Grid(dim, 2 if dim == 3 else 3, 3, 0.02)
    rng = np.random.default_rng(11)
    u0, du0, lamN = 0.3 * rng.standard_normal((3, dim) + g.global_shape())
    _, traj = ork.rk_forward(g.rhs, u0, 2e-3, 5, scheme)
    duN = ork.rk_tangent(g.jac, traj, du0, 2e-3, scheme)
    lam0 = ork.rk_adjoint(g.jacT, traj, lamN, 2e-3, scheme)
    a, b = np.sum(lamN * duN), np.sum(lam0 * du0)
    assert abs(a - b) < 1e-12 * np.linalg.norm(lamN) * np.linalg.norm(duN) * 10


def test_gradient_matches_finite_differences_with_second_order_taylor_remainder():
    g = Grid(2, 2, 4, 0.02)
    rng = np.random.default_rng(12)
    u0, uo, du = 0.5 * rng.standard_normal((3, 2) + g.global_shape())
    J0, lam0, _ = ork.objective_and_gradient(g, u0, uo, 1e-3, 8, "ssprk3")
    slope = np.sum(lam0 * du)
    rem = []
    for eps in (1e-1, 1e-2, 1e-3):
        J1 = ork.objective_and_gradient(g, u0 + eps * du, uo, 1e-3, 8, "ssprk3")[0]
        rem.append(abs(J1 - J0 - eps * slope))
    # remainder O(eps^2): each decade drops it by ~100
    assert rem[1] < rem[0] / 50 and rem[2] < rem[1] / 50
    fd = (ork.objective_and_gradient(g, u0 + 1e-5 * du, uo, 1e-3, 8, "ssprk3")[0]
          - ork.objective_and_gradient(g, u0 - 1e-5 * du, uo, 1e-3, 8, "ssprk3")[0]) / 2e-5
    assert abs(fd - slope) < 1e-7 * abs(slope)   # the paper reports ~7 digits (Sec. 6)


# ------------------------------------------------ binomial checkpointing (Sec. 5.3)
def test_dp_optimum_is_griewanks_binomial_count():
    """P(l, s) with s free slots beyond the stored start equals r l - C(s'+r, s'+1), s' = s+1 snapshots."""
    for l in range(1, 45):
        for s in range(1, 6):
            sp = s + 1
            r = 0
            while comb(sp + r, sp) < l:
                r += 1
            assert optimal_advances(l, s) == r * l - comb(sp + r, sp + 1)


@pytest.mark.parametrize("nsteps,slots", [(1, 1), (7, 1), (12, 2), (20, 3), (30, 4), (9, 0)])
def test_checkpointed_gradient_equals_store_all_bitwise(nsteps, slots):
    g = Grid(1, 3, 3, 0.05)
    rng = np.random.default_rng(13)
    u0, lamT = rng.standard_normal((2, 1) + g.global_shape())
    _, traj = ork.rk_forward(g.rhs, u0, 1e-2, nsteps, "rk4")
    ref = ork.rk_adjoint(g.jacT, traj, lamT, 1e-2, "rk4")
    got, count = checkpointed_gradient_lam0(g.rhs, g.jacT, u0, lamT, 1e-2, nsteps, "rk4", slots)
    assert np.array_equal(got, ref)
    assert count == optimal_advances(nsteps, slots)


# ------------------------------------------------ Crank-Nicolson (Sec. 6.3, implicit scheme)
from oracle import cn as ocn


def test_cn_step_is_the_1_1_pade_approximant_on_linear_problems():
    """For F(u) = A u one CN step is (I - dt A/2)^-1 (I + dt A/2) u, and its adjoint the transpose."""
    rng = np.random.default_rng(21)
    A = rng.standard_normal((7, 7))
    dt = 0.2
    u = rng.standard_normal(7)
    un, _ = ocn.cn_step(lambda y: A @ y, lambda y, w: A @ w, u, dt)
    R = np.linalg.solve(np.eye(7) - 0.5 * dt * A, np.eye(7) + 0.5 * dt * A)
    assert np.max(np.abs(un - R @ u)) < 1e-13 * np.max(np.abs(R @ u))
    lam = rng.standard_normal(7)
    back = ocn.cn_adjoint(lambda y: A.T, [u, un], lam, dt)
    assert np.max(np.abs(back - R.T @ lam)) < 1e-13 * np.max(np.abs(R.T @ lam))


def test_cn_step_satisfies_its_residual_and_is_second_order():
    g = Grid(1, 16, 9, 0.05, L=4.0)
    x = g.coords()

    def exact(t):
        e = np.exp(-0.05 * t * np.pi ** 2)
        return (2 * 0.05 * np.pi * np.sin(np.pi * x) * e / (2 + e * np.cos(np.pi * x)))[None]

    errs = []
    for steps in (10, 20):
        uT, traj = ocn.cn_forward(g.rhs, g.jac, exact(0.0), 0.4 / steps, steps)
        errs.append(np.max(np.abs(uT - exact(0.4))))
        u0, u1 = traj[0], traj[1]
        R = u1 - u0 - 0.5 * (0.4 / steps) * (g.rhs(u0) + g.rhs(u1))
        assert np.max(np.abs(R)) < 1e-14
    assert 3.0 < errs[0] / errs[1] < 5.0        # second order in time


def test_cn_tangent_adjoint_duality_and_gradient():
    g = Grid(2, 2, 3, 0.02)
    rng = np.random.default_rng(22)
    u0, du0, uo = 0.3 * rng.standard_normal((3, 2) + g.global_shape())
    dt, steps = 5e-3, 4
    uN, traj = ocn.cn_forward(g.rhs, g.jac, u0, dt, steps)
    Jd = lambda u: ocn.assembled_jacobian(g.jac, u)
    lamN = rng.standard_normal(u0.shape)
    duN = ocn.cn_tangent(Jd, traj, du0, dt)
    lam0 = ocn.cn_adjoint(lambda u: Jd(u).T, traj, lamN, dt)
    assert abs(np.sum(lamN * duN) - np.sum(lam0 * du0)) < 1e-11 * np.linalg.norm(lamN) * np.linalg.norm(duN)
    J0, grad, _ = ocn.cn_objective_and_gradient(g, u0, uo, dt, steps)
    eps = 1e-5
    fd = (ocn.cn_objective_and_gradient(g, u0 + eps * du0, uo, dt, steps)[0]
          - ocn.cn_objective_and_gradient(g, u0 - eps * du0, uo, dt, steps)[0]) / (2 * eps)
    assert abs(fd - np.sum(grad * du0)) < 1e-7 * abs(fd)


@pytest.mark.parametrize("N,tol", [(4, 2e-2), (6, 1e-3), (8, 1e-5)])
def test_frozen_advection_sweep_converges_to_advection_diffusion_solution(N, tol):
    """Sec. 6.1 convergence study: with the advection frozen at a constant speed a,
    du/dt = J(a) u is u_t + a u_x = nu u_xx, whose solution translates and damps
    each Fourier mode (closed form in inputs.advection_diffusion_1d)."""
    nu, a, T = 1e-3, 0.1, 0.05
    g = Grid(1, 8, N, nu, L=1.0)
    x = g.coords()
    c = inputs.advection_diffusion_coefs(5)
    A = np.full((1, g.G), a)
    steps = 100
    uT, _ = ork.rk_forward(lambda u: g.jac(A, u), inputs.advection_diffusion_1d(x, 0.0, c, nu, a), T / steps,
                           steps, "rk4")
    ref = inputs.advection_diffusion_1d(x, T, c, nu, a)
    assert np.max(np.abs(uT - ref)) < tol
    # a wrong sign of the advection would move the modes the other way
    assert np.max(np.abs(ref - inputs.advection_diffusion_1d(x, T, c, nu, -a))) > 0.1


# ----------------------------------------------------- adaptive stepping (Sec. 5.1)
def test_bs3_embedded_pair_orders():
    """For u' = a u (z = a dt) the stages are k1 = a u, k2 = a (1 + z/2) u,
    k3 = a (1 + 3z/4 + 3z^2/8) u and k4 = a R(z) u with R = 1 + z + z^2/2 + z^3/6, so
    the companion solution is (1 + z + z^2/2 + 3z^3/16 + z^4/48) u and the error
    estimate E = u_{n+1} - uhat_{n+1} is exactly -(z^3 + z^4)/48 u: O(dt^3), the
    local error of the second-order member."""
    a = -1.3
    for dt in (1e-2, 5e-3, 0.3):
        _, _, E = oad.bs3_step(lambda y: a * y, np.array([1.0]), dt)
        z = a * dt
        assert abs(E[0] + (z ** 3 + z ** 4) / 48.0) < 1e-15 * max(1.0, abs(z) ** 3)


def test_adaptive_sweep_hits_the_horizon_and_follows_the_tolerance():
    a = -2.0
    errs = []
    for tol in (1e-5, 1e-8):
        u, traj, dts, rej = oad.adaptive_forward(lambda y: a * y, np.array([1.0]), 1.0, 0.3, tol, tol)
        assert abs(sum(dts) - 1.0) < 1e-13
        errs.append(abs(u[0] - np.exp(a)))
    assert errs[1] < errs[0] / 100
    # a large first step is rejected and shrunk
    _, _, dts, rej = oad.adaptive_forward(lambda y: a * y, np.array([1.0]), 1.0, 0.9, 1e-8, 1e-8)
    assert rej >= 1 and dts[0] < 0.9


def test_adaptive_adjoint_is_the_transpose_of_its_tangent():
    g = Grid(1, 6, 5, 0.02)
    rng = np.random.default_rng(21)
    u0 = inputs.field_1d(g.coords(), 1)
    _, traj, dts, _ = oad.adaptive_forward(g.rhs, u0, 0.2, 0.01, 1e-6, 1e-6)
    assert len(set(dts)) > 2                     # the step really varies
    du0, lamT = rng.standard_normal((2,) + u0.shape)
    duN = oad.tangent_variable(g.jac, traj, du0, dts)
    lam0 = oad.adjoint_variable(g.jacT, traj, lamT, dts)
    lhs, rhs = float(np.sum(lamT * duN)), float(np.sum(lam0 * du0))
    assert abs(lhs - rhs) < 1e-12 * max(abs(lhs), 1.0)
