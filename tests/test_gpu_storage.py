"""Two-level trajectory store (device + pinned host memory) on the GPU.

States that do not fit the device budget go to pinned host memory through a
staging ring on a second stream; the arithmetic is that of SEM_CKPT_STATES, so
the gradients are bitwise equal to it.
"""
import time

import numpy as np
import pytest
import torch

from paper_1806_01422_gb300 import Sem, inputs
from paper_1806_01422_gb300 import _lib as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1806_01422_gb300 import build
    build.build()


def _fields(s):
    x = s.coords()
    return inputs.workload_field(s.dim, x, 1), inputs.workload_field(s.dim, x, 2)


@pytest.mark.parametrize("prec", ["fp64", "fp32_bulk"])
@pytest.mark.parametrize("dev_states", [0, 5, 19])
def test_two_level_gradient_is_bitwise_equal_to_states(prec, dev_states):
    dim, E, N, nu, dt, steps = 2, 4, 5, 1e-3, 2e-3, 20
    ref = Sem(dim, E, N, nu, precision=prec, ckpt="states")
    vb = ref.ndof * 8
    s = Sem(dim, E, N, nu, precision=prec, ckpt="two_level", ckpt_budget_bytes=(dev_states + 3) * vb)
    s.set_host_tier(steps * vb)
    u0, uo = _fields(s)
    J0, g0 = ref.objective_grad(u0, uo, dt, steps, "rk4")
    J1, g1 = s.objective_grad(u0, uo, dt, steps, "rk4")
    info = s.trajectory_info()
    assert info["mode"] == "two_level" and info["device"] == dev_states and info["host"] == steps - dev_states
    assert J0 == J1 and torch.equal(g0, g1)
    # the same through the separate sweeps, with the graph switch on (the host tier is never captured)
    s.use_graph(True)
    J2, g2 = s.objective_grad(u0, uo, dt, steps, "rk4")
    assert J2 == J0 and torch.equal(g2, g0) and s.graph_replays() == 0
    uT = s.rk_forward(u0, dt, steps, "ssprk3")
    lam = s.rk_adjoint(uT)
    uT0 = ref.rk_forward(u0, dt, steps, "ssprk3")
    assert torch.equal(uT, uT0) and torch.equal(lam, ref.rk_adjoint(uT0))


def test_auto_mode_picks_two_level_after_states():
    dim, E, N, nu, dt, steps = 2, 4, 5, 1e-3, 2e-3, 20
    s = Sem(dim, E, N, nu, ckpt="auto", ckpt_budget_bytes=10 * 2 * 400 * 8)
    u0, uo = _fields(s)
    s.objective_grad(u0, uo, dt, steps, "rk4")
    assert s.trajectory_info()["mode"] == "binomial"      # no host tier yet
    s.set_host_tier(1 << 20)
    s.objective_grad(u0, uo, dt, steps, "rk4")
    info = s.trajectory_info()
    assert info["mode"] == "two_level" and info["device"] == 7 and info["host"] == 13


def test_two_level_errors():
    s = Sem(2, 4, 5, 1e-3, ckpt="two_level", ckpt_budget_bytes=8 * 6400)
    u0, uo = _fields(s)
    with pytest.raises(L.SemError) as e:             # no host budget
        s.objective_grad(u0, uo, 2e-3, 20, "rk4")
    assert e.value.code == L.SEM_ERR_ARG
    s.set_host_tier(2 * 6400)                         # 15 host states needed
    with pytest.raises(L.SemError) as e:
        s.objective_grad(u0, uo, 2e-3, 20, "rk4")
    assert e.value.code == L.SEM_ERR_OOM
    s.set_host_tier(0)


def test_two_level_copies_overlap_the_sweeps():
    """64x64 quads, N=7 (3.2 MB states), 300 RK4 steps with 225 of the states in host memory."""
    dim, E, N, nu, dt, steps = 2, 64, 7, 1e-3, 2e-4, 300
    ref = Sem(dim, E, N, nu, ckpt="states")
    vb = ref.ndof * 8
    s = Sem(dim, E, N, nu, ckpt="two_level", ckpt_budget_bytes=(75 + 3) * vb)
    s.set_host_tier(steps * vb)
    u0, uo = _fields(s)
    t = {}
    for name, h in (("states", ref), ("two_level", s)):
        h.objective_grad(u0, uo, dt, steps, "rk4")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            J, g = h.objective_grad(u0, uo, dt, steps, "rk4")
        torch.cuda.synchronize()
        t[name] = (time.perf_counter() - t0) / 3
    print("gradient evaluation: states %.1f ms, two-level %.1f ms" % (1e3 * t["states"], 1e3 * t["two_level"]))
    assert s.trajectory_info()["host"] == 225
    assert t["two_level"] < 1.5 * t["states"]
