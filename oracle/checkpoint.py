"""Binomial checkpointing by brute force.  TEST INFRASTRUCTURE ONLY.

Sec. 5.3 of arXiv:1806.01422: the adjoint sweep needs every forward state in
reverse order; storing all of them may not fit, and the optimal trade between
stored and recomputed states for a known number of steps and slots is given by
the revolve algorithm of Griewank and Walther.

This module computes that optimum by exhaustive dynamic programming over the
first split point, which is the definition of "optimal" written out:

  P(1, s) = 0,   P(l, 0) = l (l - 1) / 2,
  P(l, s) = min_{1 <= m < l} [ m + P(l - m, s - 1) + P(m, s) ],

where P(l, s) counts the forward steps (advances) needed to reverse l steps that
start from a stored state with s further free slots; reversing a single step
is one taped forward step plus its adjoint step and is not counted.  It also
replays the recursion to produce the checkpointed adjoint gradient, which must
equal the store-all gradient exactly.
"""
from functools import lru_cache

from .rk import rk_step, rk_adjoint_step


def optimal_advances(l, s):
    """P(l, s) of the module docstring (exhaustive DP)."""
    @lru_cache(maxsize=None)
    def P(l, s):
        if l <= 1:
            return 0
        if s == 0:
            return l * (l - 1) // 2
        return min(m + P(l - m, s - 1) + P(m, s) for m in range(1, l))
    return P(l, s)


def checkpointed_gradient_lam0(F, JT, u0, lamT, dt, nsteps, scheme, slots):
    """Reverse ``nsteps`` steps from u0 with ``slots`` free state slots (DP-optimal splits).

    Returns (lam_0, number of advances used).  Advances count plain forward
    steps; every reversed step additionally runs one taped forward step.
    """
    @lru_cache(maxsize=None)
    def best(l, s):
        if l <= 1:
            return 0, 0
        if s == 0:
            return l * (l - 1) // 2, 0
        return min((m + best(l - m, s - 1)[0] + best(m, s)[0], m) for m in range(1, l))

    count = [0]

    def advance(u, k):
        for _ in range(k):
            u, _ = rk_step(F, u, dt, scheme)
            count[0] += 1
        return u

    def reverse(u_start, l, s, lam):
        # u_start is the stored state at the start of the range
        if l == 1:
            _, Y = rk_step(F, u_start, dt, scheme)
            return rk_adjoint_step(JT, Y, lam, dt, scheme)
        if s == 0:
            for k in range(l - 1, -1, -1):
                u = advance(u_start.copy(), k)
                _, Y = rk_step(F, u, dt, scheme)
                lam = rk_adjoint_step(JT, Y, lam, dt, scheme)
            return lam
        m = best(l, s)[1]
        u_mid = advance(u_start.copy(), m)
        lam = reverse(u_mid, l - m, s - 1, lam)
        return reverse(u_start, m, s, lam)

    lam0 = reverse(u0.copy(), nsteps, slots, lamT.copy())
    return lam0, count[0]
