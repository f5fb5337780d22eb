"""Data assimilation: recover u0 from a final-time observation (Fig. 1 loop, Sec. 5.5).

Each L-BFGS iteration evaluates the misfit J(u0) = 1/2 ||u_N(u0) - u_obs||_M^2 and
its gradient with one forward sweep and one discrete-adjoint sweep on the GPU
(sem_objective_grad); the quasi-Newton update and the Moré-Thuente line
search run on device tensors in FP64.
"""
from .lbfgs import lbfgs


def recover_initial_condition(sem, u_obs, u_init, dt, nsteps, scheme="rk4", iters=30, m=8, callback=None):
    """Return (u0 estimate, history [(iteration, J, |grad|, evaluations)])."""
    u_obs = sem._dev(u_obs, "u_obs")
    grad = sem.empty()

    def fg(x):
        J, g = sem.objective_grad(x, u_obs, dt, nsteps, scheme, grad=grad)
        return J, g

    x0 = sem._dev(u_init, "u_init").clone()
    return lbfgs(fg, x0, m=m, max_iter=iters, gtol=1e-12, callback=callback)
