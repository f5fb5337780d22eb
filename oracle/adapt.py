"""Adaptive time stepping for the explicit sweep.  TEST INFRASTRUCTURE ONLY.

Sec. 5.1 of arXiv:1806.01422 lets PETSc choose the step from an estimate of the
local truncation error, weighted by absolute and relative tolerances.  The paper
names neither the embedded pair nor the controller; the reading used on both
sides of the parity tests is:

* pair: Bogacki-Shampine 3(2) (Bogacki & Shampine, Appl. Math. Lett. 2 (1989)):
  the third-order solution u_{n+1} = u_n + dt (2/9 k1 + 1/3 k2 + 4/9 k3) with
  k1 = F(u_n), k2 = F(u_n + dt/2 k1), k3 = F(u_n + 3/4 dt k2), and the
  second-order companion with weights (7/24, 1/4, 1/3, 1/8) on (k1, k2, k3, k4),
  k4 = F(u_{n+1});
* error: E = dt sum_i (b_i - bhat_i) k_i, measured in the weighted RMS norm
  err = sqrt(mean_i (E_i / (atol + rtol max(|u_n,i|, |u_{n+1},i|)))^2);
* controller (Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4): accept when
  err <= 1; the next trial step is dt min(fmax, max(fmin, 0.9 err^(-1/3))) with
  fmin = 0.2, fmax = 5, and fmax = 1 right after a rejection; a step that would
  pass the horizon T is shortened to end on it.
* adjoint: the accepted steps are differentiated with their step sizes held
  fixed (the controller's dependence on u0 is not differentiated).
"""
import numpy as np

from . import rk

B_HAT = np.array([7.0 / 24.0, 1.0 / 4.0, 1.0 / 3.0, 1.0 / 8.0])
SAFETY, FMIN, FMAX = 0.9, 0.2, 5.0


def bs3_step(F, u, dt):
    """One Bogacki-Shampine step: (u_{n+1}, stage values [Y1, Y2, Y3], error vector E)."""
    A, b = rk.TABLEAUX["bs3"]
    Y, k = [], []
    for i in range(3):
        Yi = u.copy()
        for j in range(i):
            if A[i, j] != 0.0:
                Yi = Yi + dt * A[i, j] * k[j]
        Y.append(Yi)
        k.append(F(Yi))
    un = u.copy()
    for i in range(3):
        un = un + dt * b[i] * k[i]
    k.append(F(un))
    E = np.zeros_like(u)
    for i in range(4):
        bi = b[i] if i < 3 else 0.0
        E = E + dt * (bi - B_HAT[i]) * k[i]
    return un, Y, E


def wrms(E, u0, u1, atol, rtol):
    w = atol + rtol * np.maximum(np.abs(u0), np.abs(u1))
    return float(np.sqrt(np.mean((E / w) ** 2)))


def adaptive_forward(F, u0, T, dt0, atol, rtol, max_steps=100000):
    """Integrate to T; returns (u_T, stage trajectory, accepted step sizes, rejected count)."""
    u = np.array(u0, dtype=np.float64, copy=True)
    t, dt = 0.0, dt0
    traj, dts, rejected = [], [], 0
    after_reject = False
    while t < T and len(dts) < max_steps:
        last = t + dt >= T * (1.0 - 1e-12)
        h = T - t if last else dt
        un, Y, E = bs3_step(F, u, h)
        err = wrms(E, u, un, atol, rtol)
        fmax = 1.0 if after_reject else FMAX
        fac = min(fmax, max(FMIN, SAFETY * err ** (-1.0 / 3.0))) if err > 0 else fmax
        if err <= 1.0:
            traj.append(Y)
            dts.append(h)
            u = un
            t = T if last else t + h
            after_reject = False
            dt = h * fac if not last else dt
        else:
            rejected += 1
            after_reject = True
            dt = h * fac
    return u, traj, dts, rejected


def adjoint_variable(JT, traj, lamT, dts):
    """Backward sweep of the accepted BS3 steps with their step sizes held fixed."""
    lam = np.array(lamT, dtype=np.float64, copy=True)
    for Y, h in zip(reversed(traj), reversed(dts)):
        lam = rk.rk_adjoint_step(JT, Y, lam, h, "bs3")
    return lam


def tangent_variable(Jv, traj, du0, dts):
    du = np.array(du0, dtype=np.float64, copy=True)
    for Y, h in zip(traj, dts):
        du = rk.rk_tangent(Jv, [Y], du, h, "bs3")
    return du
