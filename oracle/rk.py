"""Explicit Runge-Kutta forward sweep and its discrete adjoint.  TEST INFRASTRUCTURE ONLY.

Sec. 4.1 of arXiv:1806.01422 writes an explicit step as u_{n+1} = A(u_n, P[u_n]),
builds the discrete Lagrangian with the M-weighted inner product, and obtains the
adjoint recursion (eq. adjointloop), its terminal condition (eq. initadj) and the
gradient (eq. gradient); eq. adjtime differentiates A through both arguments.
The paper works the forward-Euler case out and defers multistage methods to the
PETSc adjoint papers; here the same Lagrangian argument is carried through the
stages of an explicit Butcher tableau:

forward   Y_i = u_n + dt sum_{j<i} a_ij k_j,   k_i = F(Y_i),
          u_{n+1} = u_n + dt sum_i b_i k_i;
adjoint   for i = s..1:  nu_i = dt (b_i lam_{n+1} + sum_{j>i} a_ji mu_j),
                         mu_i = J(Y_i)^T nu_i;
          lam_n = lam_{n+1} + sum_i mu_i.

lam are Euclidean adjoints (lam_N = dJ/du_N); the paper's M-weighted adjoint is
v_n = M^-1 lam_n.  Forward Euler (s = 1, b = 1) reproduces the paper's
v_n = v_{n+1} + dt J^T v_{n+1} up to that M scaling.
"""
import numpy as np

# Butcher tableaux (A strictly lower triangular, b weights).
TABLEAUX = {
    # classic fourth-order Runge-Kutta
    "rk4": (np.array([[0.0, 0.0, 0.0, 0.0],
                      [0.5, 0.0, 0.0, 0.0],
                      [0.0, 0.5, 0.0, 0.0],
                      [0.0, 0.0, 1.0, 0.0]]),
            np.array([1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0])),
    # Shu-Osher strong-stability-preserving third-order method, Butcher form
    "ssprk3": (np.array([[0.0, 0.0, 0.0],
                         [1.0, 0.0, 0.0],
                         [0.25, 0.25, 0.0]]),
               np.array([1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0])),
    # forward Euler, the case worked out in Sec. 4.1
    "euler": (np.array([[0.0]]), np.array([1.0])),
    # Bogacki-Shampine third-order method (the solution part of the 3(2) pair; its
    # fourth, first-same-as-last stage only serves the error estimate, oracle/adapt.py)
    "bs3": (np.array([[0.0, 0.0, 0.0],
                      [0.5, 0.0, 0.0],
                      [0.0, 0.75, 0.0]]),
            np.array([2.0 / 9.0, 1.0 / 3.0, 4.0 / 9.0])),
}


def rk_step(F, u, dt, scheme):
    """One explicit RK step; returns (u_{n+1}, [Y_1..Y_s])."""
    A, b = TABLEAUX[scheme]
    s = len(b)
    Y, k = [], []
    for i in range(s):
        Yi = u.copy()
        for j in range(i):
            if A[i, j] != 0.0:
                Yi = Yi + dt * A[i, j] * k[j]
        Y.append(Yi)
        k.append(F(Yi))
    out = u.copy()
    for i in range(s):
        out = out + dt * b[i] * k[i]
    return out, Y


def rk_forward(F, u0, dt, nsteps, scheme):
    """Forward sweep storing every stage of every step (store-all trajectory)."""
    u = np.array(u0, dtype=np.float64, copy=True)
    traj = []
    for _ in range(nsteps):
        u, Y = rk_step(F, u, dt, scheme)
        traj.append(Y)
    return u, traj


def rk_adjoint_step(JT, Y, lam, dt, scheme):
    """Discrete adjoint of one step given its stage values Y (see module docstring)."""
    A, b = TABLEAUX[scheme]
    s = len(b)
    mu = [None] * s
    for i in range(s - 1, -1, -1):
        nu_i = dt * b[i] * lam
        for j in range(i + 1, s):
            if A[j, i] != 0.0:
                nu_i = nu_i + dt * A[j, i] * mu[j]
        mu[i] = JT(Y[i], nu_i)
    out = lam.copy()
    for i in range(s):
        out = out + mu[i]
    return out


def rk_adjoint(JT, traj, lamT, dt, scheme):
    """Backward sweep over a stored trajectory: lam_0 from lam_N."""
    lam = np.array(lamT, dtype=np.float64, copy=True)
    for Y in reversed(traj):
        lam = rk_adjoint_step(JT, Y, lam, dt, scheme)
    return lam


def rk_tangent(Jv, traj, du0, dt, scheme):
    """Tangent-linear sweep: du_N = (d u_N / d u_0) du0 along a stored trajectory."""
    A, b = TABLEAUX[scheme]
    s = len(b)
    du = np.array(du0, dtype=np.float64, copy=True)
    for Y in traj:
        dk = []
        for i in range(s):
            dY = du.copy()
            for j in range(i):
                if A[i, j] != 0.0:
                    dY = dY + dt * A[i, j] * dk[j]
            dk.append(Jv(Y[i], dY))
        for i in range(s):
            du = du + dt * b[i] * dk[i]
    return du


def objective_and_gradient(grid, u0, u_obs, dt, nsteps, scheme):
    """Misfit J(u0) = 1/2 ||u_N - u_obs||_M^2 and its Euclidean gradient lam_0 (Fig. 1 workflow)."""
    uN, traj = rk_forward(grid.rhs, u0, dt, nsteps, scheme)
    J, lamN = grid.objective(uN, u_obs)
    lam0 = rk_adjoint(grid.jacT, traj, lamN, dt, scheme)
    return J, lam0, uN
