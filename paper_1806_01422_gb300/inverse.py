"""Data assimilation: recover u0 from a final-time observation (Fig. 1 loop, Sec. 5.5).

Each L-BFGS iteration evaluates the misfit J(u0) = 1/2 ||u_N(u0) - u_obs||_M^2 and
its gradient with one forward sweep and one discrete-adjoint sweep on the GPU
(sem_objective_grad); the quasi-Newton update and the strong-Wolfe line
search run on device tensors in FP64.
"""
from . import _lib as L
from .lbfgs import lbfgs


def mass_diagonal(sem):
    """The diagonal of the global GLL mass matrix M: the misfit adjoint M (u - u_obs) at u - u_obs = 1."""
    ones = sem.empty().fill_(1.0)
    lam = sem.empty()
    sem.objective(ones, ones.new_zeros(ones.shape), lam)
    return lam


def recover_initial_condition(sem, u_obs, u_init, dt, nsteps, scheme="rk4", iters=30, m=8, callback=None,
                              precondition=True):
    """Return (u0 estimate, history [(iteration, J, |grad|, evaluations)]).

    The misfit weights the nodes by the GLL mass, whose entries differ by up to
    (w_mid / w_end)^d between the middle and the corners of an element, so the
    Euclidean gradient is badly scaled.  With precondition=True L-BFGS starts from
    H_0 = M^-1 (the paper's M-weighted adjoint v = M^-1 lam, Sec. 4.1): for a short
    horizon the misfit's Hessian is close to M and the first step is close to Newton's.
    """
    u_obs = sem._dev(u_obs, "u_obs")
    grad = sem.empty()
    h0 = 1.0 / mass_diagonal(sem) if precondition else None

    def fg(x):
        try:
            J, g = sem.objective_grad(x, u_obs, dt, nsteps, scheme, grad=grad)
        except L.SemError as e:
            if e.code != L.SEM_ERR_NONFINITE:
                raise
            return float("inf"), None   # a trial point where the forward sweep diverges
        return J, g

    x0 = sem._dev(u_init, "u_init").clone()
    return lbfgs(fg, x0, m=m, max_iter=iters, gtol=1e-12, callback=callback, h0_diag=h0)
