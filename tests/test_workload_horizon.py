"""Why the 3D workloads stop at 300 RK steps, checked with the oracle on the CPU.

The seeded k^-5/3 field of the 3D workloads steepens under Burgers into fronts
about nu / max|u| wide, far below the grid spacing at nu = 5e-4.  GLL
collocation without over-integration (the paper's discretisation, Sec. 3.2) has
nothing that damps the aliasing this produces, and the discrete solution
diverges.  On the full 32^3-element grid this happens between steps 400 and 500
(max|u| 0.99 at step 300, 1.08 at 400, non-finite by 500).  Here the oracle shows
the same mechanism on a 4^3-element grid of the same order, viscosity and step:
the field stays bounded near its initial max|u| = 1 for the first hundred steps,
then grows without bound and becomes non-finite before step 500.
"""
import numpy as np

from oracle.sem import Grid
from oracle import rk as ork
from paper_1806_01422_gb300 import inputs


def test_3d_workload_field_diverges_on_an_under_resolved_grid():
    g = Grid(3, 4, 7, 5e-4)
    u = inputs.workload_field(3, g.coords(), inputs.SEED_U0)
    assert abs(np.max(np.abs(u)) - 1.0) < 1e-12
    peak = {}
    with np.errstate(all="ignore"):
        for n in range(1, 501):
            u, _ = ork.rk_step(g.rhs, u, 2.5e-4, "rk4")
            m = float(np.max(np.abs(u)))
            peak[n] = m
            if not np.isfinite(m):
                break
    assert max(peak[n] for n in range(1, 101)) < 1.05          # bounded while the fronts form
    assert peak[300] > 1.1                                       # growing past the initial amplitude
    last = max(peak)
    assert last < 500 and not np.isfinite(peak[last])            # non-finite before step 500
