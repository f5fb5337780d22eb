"""Limited-memory BFGS with a Moré-Thuente line search (the optimizer of Sec. 5.5).

Sec. 5.5 of arXiv:1806.01422 drives the optimisation with TAO's LMVM method: a
limited-memory quasi-Newton direction d_k = -H_k grad f(x_k) from the last m
(s, y) pairs, then a Moré-Thuente line search for a step that satisfies the
strong Wolfe conditions.  This module implements both from their published
descriptions (Nocedal & Wright, Numerical Optimization, Alg. 7.4 two-loop
recursion; Moré & Thuente, ACM TOMS 20 (1994), the safeguarded cubic/quadratic
step on an interval of uncertainty).  Vectors are torch tensors (float64, on
the GPU for the SEM problems); the objective callback returns (f, grad).
"""
import math

import torch


def _dot(a, b):
    return float(torch.dot(a.reshape(-1), b.reshape(-1)))


def _cstep(stx, fx, dx, sty, fy, dy, stp, fp, dp, brackt, stpmin, stpmax):
    """One safeguarded step of the Moré-Thuente interval update.

    (stx, fx, dx): best step so far, (sty, fy, dy): other end of the interval,
    (stp, fp, dp): trial step; f values and derivatives along the direction.
    Returns the updated (stx, fx, dx, sty, fy, dy, new trial step, brackt).
    """
    sgnd = dp * (dx / abs(dx)) if dx != 0.0 else dp
    if fp > fx:
        # higher function value: the minimiser is bracketed; cubic vs quadratic step
        theta = 3.0 * (fx - fp) / (stp - stx) + dx + dp
        s = max(abs(theta), abs(dx), abs(dp))
        gamma = s * math.sqrt(max(0.0, (theta / s) ** 2 - (dx / s) * (dp / s)))
        if stp < stx:
            gamma = -gamma
        p = (gamma - dx) + theta
        q = ((gamma - dx) + gamma) + dp
        stpc = stx + (p / q) * (stp - stx)
        stpq = stx + ((dx / ((fx - fp) / (stp - stx) + dx)) / 2.0) * (stp - stx)
        stpf = stpc if abs(stpc - stx) < abs(stpq - stx) else stpc + (stpq - stpc) / 2.0
        brackt = True
    elif sgnd < 0.0:
        # derivatives of opposite sign: bracketed
        theta = 3.0 * (fx - fp) / (stp - stx) + dx + dp
        s = max(abs(theta), abs(dx), abs(dp))
        gamma = s * math.sqrt(max(0.0, (theta / s) ** 2 - (dx / s) * (dp / s)))
        if stp > stx:
            gamma = -gamma
        p = (gamma - dp) + theta
        q = ((gamma - dp) + gamma) + dx
        stpc = stp + (p / q) * (stx - stp)
        stpq = stp + (dp / (dp - dx)) * (stx - stp)
        stpf = stpc if abs(stpc - stp) > abs(stpq - stp) else stpq
        brackt = True
    elif abs(dp) < abs(dx):
        # same sign, derivative magnitude decreases
        theta = 3.0 * (fx - fp) / (stp - stx) + dx + dp
        s = max(abs(theta), abs(dx), abs(dp))
        gamma = s * math.sqrt(max(0.0, (theta / s) ** 2 - (dx / s) * (dp / s)))
        if stp > stx:
            gamma = -gamma
        p = (gamma - dp) + theta
        q = (gamma + (dx - dp)) + gamma
        r = p / q
        stpc = stp + r * (stx - stp) if (r < 0.0 and gamma != 0.0) else (stpmax if stp > stx else stpmin)
        stpq = stp + (dp / (dp - dx)) * (stx - stp)
        if brackt:
            stpf = stpc if abs(stpc - stp) < abs(stpq - stp) else stpq
            stpf = min(stp + 0.66 * (sty - stp), stpf) if stp > stx else max(stp + 0.66 * (sty - stp), stpf)
        else:
            stpf = stpc if abs(stpc - stp) > abs(stpq - stp) else stpq
            stpf = min(stpmax, max(stpmin, stpf))
    else:
        # same sign, derivative magnitude does not decrease
        if brackt:
            theta = 3.0 * (fp - fy) / (sty - stp) + dy + dp
            s = max(abs(theta), abs(dy), abs(dp))
            gamma = s * math.sqrt(max(0.0, (theta / s) ** 2 - (dy / s) * (dp / s)))
            if stp > sty:
                gamma = -gamma
            p = (gamma - dp) + theta
            q = ((gamma - dp) + gamma) + dy
            stpf = stp + (p / q) * (sty - stp)
        else:
            stpf = stpmax if stp > stx else stpmin
    # update the interval of uncertainty
    if fp > fx:
        sty, fy, dy = stp, fp, dp
    else:
        if sgnd < 0.0:
            sty, fy, dy = stx, fx, dx
        stx, fx, dx = stp, fp, dp
    return stx, fx, dx, sty, fy, dy, stpf, brackt


def more_thuente(phi, f0, g0, stp=1.0, ftol=1e-4, gtol=0.9, xtol=1e-10, stpmin=1e-20, stpmax=1e20, maxfev=20):
    """Step satisfying the strong Wolfe conditions for phi(t) = f(x + t d).

    phi(t) returns (f, derivative along d, payload); f0, g0 at t = 0 (g0 < 0).
    A trial step whose f or derivative is not finite (the model left its range of
    validity) becomes the new upper limit of the step and the next trial moves
    halfway back towards the best step so far.
    Returns (t, f, payload, evaluations).
    """
    if g0 >= 0.0:
        raise ValueError("not a descent direction")
    brackt, stage1 = False, True
    gtest = ftol * g0
    width, width1 = stpmax - stpmin, 2.0 * (stpmax - stpmin)
    stx, fx, gx = 0.0, f0, g0
    sty, fy, gy = 0.0, f0, g0
    best = None
    for nfev in range(1, maxfev + 1):
        if brackt:
            stmin, stmax = min(stx, sty), max(stx, sty)
        else:
            stmin, stmax = stx, stp + 4.0 * (stp - stx)
        stp = min(max(stp, stpmin), stpmax)
        if brackt and (stp <= stmin or stp >= stmax or stmax - stmin <= xtol * stmax):
            stp = stx
        f, g, payload = phi(stp)
        if not (math.isfinite(f) and math.isfinite(g)):
            stpmax = stp
            stp = stx + 0.5 * (stp - stx)
            continue
        if best is None or f < best[1]:
            best = (stp, f, payload)
        ftest = f0 + stp * gtest
        if f <= ftest and abs(g) <= gtol * (-g0):
            return stp, f, payload, nfev          # strong Wolfe conditions hold
        if brackt and stmax - stmin <= xtol * stmax:
            break
        if stage1 and f <= ftest and g >= min(ftol, gtol) * g0:
            stage1 = False
        if stage1 and f <= fx and f > ftest:
            # modified function psi(t) = phi(t) - t gtest in the first stage
            fm, fxm, fym = f - stp * gtest, fx - stx * gtest, fy - sty * gtest
            gm, gxm, gym = g - gtest, gx - gtest, gy - gtest
            stx, fxm, gxm, sty, fym, gym, stp, brackt = _cstep(stx, fxm, gxm, sty, fym, gym, stp, fm, gm, brackt,
                                                               stmin, stmax)
            fx, fy = fxm + stx * gtest, fym + sty * gtest
            gx, gy = gxm + gtest, gym + gtest
        else:
            stx, fx, gx, sty, fy, gy, stp, brackt = _cstep(stx, fx, gx, sty, fy, gy, stp, f, g, brackt,
                                                           stmin, stmax)
        if brackt:
            if abs(sty - stx) >= 0.66 * width1:
                stp = stx + 0.5 * (sty - stx)
            width1, width = width, abs(sty - stx)
    if best is None:
        raise FloatingPointError("no finite function value along the search direction")
    return best[0], best[1], best[2], maxfev


def lbfgs(fg, x0, m=8, max_iter=30, gtol=1e-8, callback=None, line_search_maxfev=20, h0_diag=None):
    """Minimise f with L-BFGS (two-loop recursion) and the Moré-Thuente line search.

    fg(x) -> (f, grad); x0: tensor.  Returns (x, history) where history holds
    (iteration, f, |grad|, function evaluations).  Stops after max_iter
    iterations or when |grad| <= gtol |grad_0|.

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

        t, fn, (xn, gn), ne = more_thuente(phi, f, dg, stp=1.0, maxfev=line_search_maxfev)
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
