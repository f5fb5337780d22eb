"""Crank-Nicolson forward step and its discrete adjoint.  TEST INFRASTRUCTURE ONLY.

Sec. 6.3 of arXiv:1806.01422 times the implicit Crank-Nicolson scheme next to
explicit RK-3: the forward step needs a nonlinear (Newton) solve, its adjoint
only linear solves with the transposed Jacobian (Sec. 3.1: the Jacobian is
needed by implicit integrators and, transposed, by the discrete adjoint).

Step n -> n+1 of du/dt = F(u):
    R(u_{n+1}) = u_{n+1} - u_n - dt/2 (F(u_n) + F(u_{n+1})) = 0,
solved by Newton's method with (I - dt/2 J(u^k)) delta = -R(u^k), each linear
system solved directly on the assembled matrix (tiny grids only).

Adjoint (the same Lagrangian argument as rk.py): d u_{n+1} / d u_n =
(I - dt/2 J_{n+1})^-1 (I + dt/2 J_n), so for lam_{n+1} = dJ/du_{n+1}
    solve (I - dt/2 J_{n+1})^T mu = lam_{n+1},   lam_n = mu + dt/2 J_n^T mu.
"""
import numpy as np


def assembled_jacobian(jac, u):
    """Dense J(u) from matrix-free products with the identity's columns."""
    n = u.size
    cols = [jac(u, np.eye(n)[k].reshape(u.shape)).ravel() for k in range(n)]
    return np.array(cols).T


def cn_step(F, jac, u, dt, tol=1e-14, maxit=30):
    """One Crank-Nicolson step by Newton's method; returns (u_{n+1}, Newton iterations)."""
    Fn = F(u)
    v = u + dt * Fn                      # explicit Euler predictor
    n = u.size
    for it in range(1, maxit + 1):
        R = v - u - 0.5 * dt * (Fn + F(v))
        A = np.eye(n) - 0.5 * dt * assembled_jacobian(jac, v)
        delta = np.linalg.solve(A, -R.ravel()).reshape(u.shape)
        v = v + delta
        if np.max(np.abs(delta)) <= tol * max(1.0, np.max(np.abs(v))):
            return v, it
    return v, maxit


def cn_forward(F, jac, u0, dt, nsteps):
    u = np.array(u0, dtype=np.float64, copy=True)
    traj = [u.copy()]
    for _ in range(nsteps):
        u, _ = cn_step(F, jac, u, dt)
        traj.append(u.copy())
    return u, traj


def cn_adjoint(jacT_dense, traj, lamT, dt):
    """lam_0 from lam_N along a stored CN trajectory; jacT_dense(u) -> J(u)^T as a matrix."""
    lam = np.array(lamT, dtype=np.float64, copy=True).ravel()
    n = lam.size
    for k in range(len(traj) - 1, 0, -1):
        A = np.eye(n) - 0.5 * dt * jacT_dense(traj[k])
        mu = np.linalg.solve(A, lam)
        lam = mu + 0.5 * dt * (jacT_dense(traj[k - 1]) @ mu)
    return lam.reshape(np.shape(lamT))


def cn_tangent(jac_dense, traj, du0, dt):
    """du_N = (d u_N / d u_0) du0 along a stored CN trajectory."""
    du = np.array(du0, dtype=np.float64, copy=True).ravel()
    n = du.size
    for k in range(1, len(traj)):
        A = np.eye(n) - 0.5 * dt * jac_dense(traj[k])
        du = np.linalg.solve(A, du + 0.5 * dt * (jac_dense(traj[k - 1]) @ du))
    return du.reshape(np.shape(du0))


def cn_objective_and_gradient(grid, u0, u_obs, dt, nsteps):
    """Misfit and its Euclidean gradient through the CN scheme (dense linear algebra)."""
    uN, traj = cn_forward(grid.rhs, grid.jac, u0, dt, nsteps)
    J, lamN = grid.objective(uN, u_obs)
    jT = lambda u: assembled_jacobian(grid.jac, u).T
    lam0 = cn_adjoint(jT, traj, lamN, dt)
    return J, lam0, uN
