"""The paper's optimisation loop on the GPU: L-BFGS over adjoint gradients
recovers an initial condition from its final-time field."""
import pytest
import torch

from paper_1806_01422_gb300 import Sem, inputs
from paper_1806_01422_gb300.inverse import recover_initial_condition

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1806_01422_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", ["fp64", "fp32_bulk"])
def test_lbfgs_recovers_initial_condition(prec):
    s = Sem(2, 8, 7, 1e-3, precision=prec)
    x = s.coords()
    u_true = torch.from_numpy(inputs.field_2d(x, 1)).cuda()
    u_obs = s.rk_forward(u_true, 2e-4, 40, "ssprk3").clone()
    u_init = torch.from_numpy(0.5 * inputs.field_2d(x, 3)).cuda()
    est, hist = recover_initial_condition(s, u_obs, u_init, 2e-4, 40, "ssprk3", iters=30)
    J0, Jn = hist[0][1], hist[-1][1]
    assert Jn < 1e-4 * J0
    assert all(b[1] <= a[1] for a, b in zip(hist, hist[1:]))
    err0 = float((u_init - u_true).norm() / u_true.norm())
    errn = float((est - u_true).norm() / u_true.norm())
    assert errn < 0.2 * err0
