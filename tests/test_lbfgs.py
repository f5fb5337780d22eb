"""L-BFGS with the strong-Wolfe line search on problems with known minimisers (CPU)."""
import math

import numpy as np
import pytest
import torch

from paper_1806_01422_gb300.lbfgs import lbfgs, wolfe_line_search


def test_line_search_satisfies_strong_wolfe_on_a_quartic():
    # phi(t) = (t - 2)^4 - t: minimiser where 4 (t - 2)^3 = 1
    phi = lambda t: ((t - 2) ** 4 - t, 4 * (t - 2) ** 3 - 1, None)
    f0, g0, _ = phi(0.0)
    t, f, _, n = wolfe_line_search(phi, f0, g0, t0=1.0, c1=1e-4, c2=0.1)
    assert f <= f0 + 1e-4 * t * g0
    assert abs(phi(t)[1]) <= 0.1 * abs(g0)


def test_quadratic_is_minimised_to_the_exact_solution():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((30, 30))
    A = torch.from_numpy(A @ A.T + 30 * np.eye(30))
    b = torch.from_numpy(rng.standard_normal(30))
    fg = lambda x: (float(0.5 * x @ A @ x - b @ x), A @ x - b)
    x, hist = lbfgs(fg, torch.zeros(30, dtype=torch.float64), m=10, max_iter=200, gtol=1e-12)
    assert torch.allclose(x, torch.linalg.solve(A, b), rtol=1e-9, atol=1e-10)
    assert all(h2[1] <= h1[1] for h1, h2 in zip(hist, hist[1:]))   # monotone decrease


def test_rosenbrock_converges():
    def fg(x):
        a, b = x[0], x[1]
        f = (1 - a) ** 2 + 100 * (b - a * a) ** 2
        g = torch.stack([-2 * (1 - a) - 400 * a * (b - a * a), 200 * (b - a * a)])
        return float(f), g
    x, hist = lbfgs(fg, torch.tensor([-1.2, 1.0], dtype=torch.float64), m=6, max_iter=200, gtol=1e-10)
    assert torch.allclose(x, torch.tensor([1.0, 1.0], dtype=torch.float64), atol=1e-6)


def test_line_search_backs_off_from_non_finite_values():
    """f(t) is only finite for t < 0.3 along the direction: the search must shrink into that range."""
    def phi(t):
        if t >= 0.3:
            return math.inf, math.nan, None
        return (t - 0.2) ** 2, 2.0 * (t - 0.2), t
    t, f, payload, nfev = wolfe_line_search(phi, 0.04, -0.4, t0=1.0)
    assert t < 0.3 and f < 0.04 and payload == t


def test_diagonal_initial_hessian_solves_a_badly_scaled_quadratic_at_once():
    """f = 1/2 sum a_i x_i^2 with a_i spread over four decades: with H_0 = diag(1/a) the first
    direction is the Newton step, so the unit step lands on the minimiser."""
    a = torch.logspace(0, 4, 50, dtype=torch.float64)
    x0 = torch.ones(50, dtype=torch.float64)
    fg = lambda x: (0.5 * float((a * x * x).sum()), a * x)
    x, hist = lbfgs(fg, x0, max_iter=3, h0_diag=1.0 / a)
    assert hist[1][1] < 1e-28 and float(x.abs().max()) < 1e-14
    _, plain = lbfgs(fg, x0, max_iter=3)
    assert plain[-1][1] > 1e-6          # the unscaled method is still far off after 3 iterations


@pytest.mark.parametrize("tmin", [0.01, 0.3, 0.9, 1.7, 7.0, 60.0])
@pytest.mark.parametrize("c2", [0.9, 0.1])
def test_line_search_zoom_and_expansion_meet_strong_wolfe(tmin, c2):
    """phi(t) = exp-shaped valley with its minimiser at tmin: the unit step overshoots (zoom) or
    undershoots (expansion); either way the returned step satisfies both strong Wolfe conditions."""
    def phi(t):
        z = t / tmin
        return z * z - 2.0 * math.log1p(z * z) * 0.25 - 2.0 * z, (2 * z - z / (1 + z * z) - 2.0) / tmin, None
    f0, g0, _ = phi(0.0)
    t, f, _, n = wolfe_line_search(phi, f0, g0, t0=1.0, c1=1e-4, c2=c2, maxfev=40)
    assert f <= f0 + 1e-4 * t * g0
    assert abs(phi(t)[1]) <= c2 * abs(g0) * (1 + 1e-12)
    assert n <= 40


def test_line_search_returns_best_decrease_when_budget_runs_out():
    """With one evaluation allowed the search returns the decreasing trial it has."""
    phi = lambda t: ((t - 3.0) ** 2 - 9.0, 2.0 * (t - 3.0), "p%g" % t)
    t, f, payload, n = wolfe_line_search(phi, 0.0, -6.0, t0=1.0, maxfev=1)
    assert n == 1 and t == 1.0 and f == -5.0 and payload == "p1"
