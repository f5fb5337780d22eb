"""Limited-memory BFGS with a strong-Wolfe line search (the optimizer of Sec. 5.5).

Sec. 5.5 of arXiv:1806.01422 drives the optimisation with TAO's LMVM method: a
limited-memory quasi-Newton direction d_k = -H_k grad f(x_k) from the last m
(s, y) pairs, then a line search for a step that satisfies the strong Wolfe
conditions (TAO's is More-Thuente's).  This module implements the two-loop
recursion (Nocedal & Wright, Numerical Optimization, Alg. 7.4) and a
bracket-and-zoom strong-Wolfe search (the same book, Alg. 3.5 and 3.6, with a
safeguarded Hermite-cubic step).  Vectors are torch tensors (float64, on the GPU
for the SEM problems); the objective callback returns (f, grad).
"""
import math

import torch


def _dot(a, b):
    return float(torch.dot(a.reshape(-1), b.reshape(-1)))


def _hermite_cubic_min(a, fa, da, b, fb, db):
    """Minimiser of the cubic that matches f and f' at a and b (Nocedal & Wright eq. 3.59), or None."""
    if a == b:
        return None
    d1 = da + db - 3.0 * (fa - fb) / (a - b)
    disc = d1 * d1 - da * db
    if not (disc >= 0.0) or not math.isfinite(disc):
        return None
    d2 = math.copysign(math.sqrt(disc), b - a)
    den = db - da + 2.0 * d2
    if den == 0.0:
        return None
    t = b - (b - a) * (db + d2 - d1) / den
    return t if math.isfinite(t) else None


class LineSearchStalled(FloatingPointError):
    """Every trial step was finite but none lowered f below f(0): f has stopped decreasing at
    rounding level along the direction."""


class _Probe:
    """One evaluated trial step: t, phi(t), phi'(t) and the caller's payload."""
    __slots__ = ("t", "f", "d", "payload")

    def __init__(self, t, f, d, payload):
        self.t, self.f, self.d, self.payload = t, f, d, payload

    @property
    def finite(self):
        return math.isfinite(self.f) and math.isfinite(self.d)


def wolfe_line_search(phi, f0, g0, t0=1.0, c1=1e-4, c2=0.9, maxfev=20, tmax=1e20):
    """Step length satisfying the strong Wolfe conditions for phi(t) = f(x + t d).

    The role of TAO's More-Thuente search in Sec. 5.5, written as the two-phase
    method of Nocedal & Wright (Numerical Optimization, 2nd ed., Alg. 3.5 and
    Alg. 3.6):

    * bracketing: from t0 the step doubles until a trial either violates
      sufficient decrease (or stops decreasing), or has a non-negative slope:
      then [previous, trial] holds a step that satisfies both conditions;
    * zoom: the bracket [lo, hi] shrinks around the minimiser of the cubic that
      matches phi and phi' at both ends, kept at least a tenth of the bracket
      away from either end (the midpoint when the cubic has no minimiser there);
      lo is always the lowest point that satisfies sufficient decrease.

    A trial whose value or slope is not finite (the model left its range of
    validity) is a step that is too long: it becomes the far end of the bracket
    and the search bisects towards lo.

    phi(t) returns (f, slope along d, payload); f0, g0 are phi(0) and phi'(0) < 0.
    Returns (t, f, payload, evaluations).  If no step satisfies both conditions
    within maxfev evaluations, the lowest finite trial below f0 is returned; if
    there is none, LineSearchStalled is raised when some trial was finite, and
    FloatingPointError when none was.
    """
    if not g0 < 0.0:
        raise ValueError("not a descent direction")
    nfev = 0
    best = None                      # lowest finite trial with f < f0
    any_finite = False

    def probe(t):
        nonlocal nfev, best, any_finite
        f, d, payload = phi(t)
        nfev += 1
        p = _Probe(t, f, d, payload)
        any_finite = any_finite or p.finite
        if p.finite and f < f0 and (best is None or f < best.f):
            best = p
        return p

    def armijo(p):
        return p.finite and p.f <= f0 + c1 * p.t * g0

    def curvature(p):
        return abs(p.d) <= c2 * abs(g0)

    def zoom(lo, hi):
        while nfev < maxfev:
            w = hi.t - lo.t
            t = None
            if hi.finite:
                t = _hermite_cubic_min(lo.t, lo.f, lo.d, hi.t, hi.f, hi.d)
            left, right = min(lo.t, hi.t) + 0.1 * abs(w), max(lo.t, hi.t) - 0.1 * abs(w)
            if t is None or not (left <= t <= right):
                t = lo.t + 0.5 * w
            if t == lo.t or t == hi.t:
                break
            p = probe(t)
            if not armijo(p) or p.f >= lo.f:
                hi = p
                continue
            if curvature(p):
                return p
            if p.d * (hi.t - lo.t) >= 0.0:
                hi = lo
            lo = p
        return None

    prev = _Probe(0.0, f0, g0, None)
    t = min(t0, tmax)
    found = None
    while nfev < maxfev:
        p = probe(t)
        if not armijo(p) or (prev.t > 0.0 and p.f >= prev.f):
            found = zoom(prev, p)
            break
        if curvature(p):
            found = p
            break
        if p.d >= 0.0:
            found = zoom(p, prev)
            break
        if t >= tmax:
            found = p
            break
        prev, t = p, min(2.0 * t, tmax)
    if found is None:
        found = best
    if found is None and any_finite:
        raise LineSearchStalled("no trial step lowered f below f(0) along the search direction")
    if found is None:
        raise FloatingPointError("no finite function value along the search direction")
    return found.t, found.f, found.payload, nfev


def lbfgs(fg, x0, m=8, max_iter=30, gtol=1e-8, callback=None, line_search_maxfev=20, h0_diag=None):
    """Minimise f with L-BFGS (two-loop recursion) and the strong-Wolfe line search.

    fg(x) -> (f, grad); x0: tensor.  Returns (x, history) where history holds
    (iteration, f, |grad|, function evaluations).  Stops after max_iter
    iterations, when |grad| <= gtol |grad_0|, or when no step along the
    quasi-Newton direction lowers f any more (rounding level).

    h0_diag: optional diagonal of the initial inverse Hessian H_0 (a tensor like x).
    Without it H_0 = gamma I (Nocedal & Wright eq. 7.20) and the first step is a unit
    step along -grad / |grad|; with it H_0 = gamma D, gamma = s^T y / y^T D y, and the
    first direction is -D grad (a preconditioned, scale-aware quasi-Newton method).
    """
    x = x0.clone()
    f, g = fg(x)
    g = g.clone()
    g0n = math.sqrt(_dot(g, g))
    S, Y, rho = [], [], []
    hist = [(0, f, g0n, 1)]
    nfev = 1
    for k in range(1, max_iter + 1):
        # two-loop recursion: d = -H g
        q = g.clone()
        alpha = []
        for s, y, r in zip(reversed(S), reversed(Y), reversed(rho)):
            a = r * _dot(s, q)
            alpha.append(a)
            q.add_(y, alpha=-a)
        if h0_diag is not None:
            q.mul_(h0_diag)
            if S:
                q.mul_(_dot(S[-1], Y[-1]) / _dot(Y[-1], h0_diag * Y[-1]))
        elif S:
            gamma = _dot(S[-1], Y[-1]) / _dot(Y[-1], Y[-1])
            q.mul_(gamma)
        else:
            q.mul_(1.0 / max(math.sqrt(_dot(g, g)), 1e-300))
        for (s, y, r), a in zip(zip(S, Y, rho), reversed(alpha)):
            b = r * _dot(y, q)
            q.add_(s, alpha=a - b)
        d = -q
        dg = _dot(d, g)
        if dg >= 0.0:               # not a descent direction: restart from (scaled) steepest descent
            S, Y, rho = [], [], []
            d = -(g * h0_diag) if h0_diag is not None else -g / max(math.sqrt(_dot(g, g)), 1e-300)
            dg = _dot(d, g)

        def phi(t):
            xt = x + t * d
            ft, gt = fg(xt)
            if gt is None or not math.isfinite(ft):
                return math.inf, math.nan, None
            gt = gt.clone()
            return ft, _dot(gt, d), (xt, gt)

        try:
            t, fn, (xn, gn), ne = wolfe_line_search(phi, f, dg, t0=1.0, maxfev=line_search_maxfev)
        except LineSearchStalled:
            break                   # f no longer decreases above rounding: x is as good as it gets
        nfev += ne
        s, y = xn - x, gn - g
        sy = _dot(s, y)
        if sy > 1e-300:
            S.append(s)
            Y.append(y)
            rho.append(1.0 / sy)
            if len(S) > m:
                S.pop(0)
                Y.pop(0)
                rho.pop(0)
        x, f, g = xn, fn, gn
        gn_norm = math.sqrt(_dot(g, g))
        hist.append((k, f, gn_norm, nfev))
        if callback:
            callback(k, x, f, gn_norm)
        if gn_norm <= gtol * g0n:
            break
    return x, hist
