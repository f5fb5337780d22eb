"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: FP64 form 1e-11 relative (max-norm over the output array); FP32-bulk
form 1e-5 relative on smooth workload fields;
gather-scatter results are bitwise reproducible run to run.
"""
import numpy as np
import pytest
import torch

from oracle.sem import Grid
from oracle import rk as ork
from oracle.checkpoint import checkpointed_gradient_lam0
from paper_1806_01422_gb300 import Sem, SemMisfit, inputs
from paper_1806_01422_gb300 import _lib as L

pytestmark = pytest.mark.gpu

RTOL64 = 1e-11
RTOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1806_01422_gb300 import build
    build.build()


def relerr(got, ref):
    got = got.detach().cpu().numpy() if isinstance(got, torch.Tensor) else np.asarray(got)
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def pair(dim, E, N, nu=0.037, L_box=None, **kw):
    return Sem(dim, E, N, nu, L_box=L_box, **kw), Grid(dim, E, N, nu, L=L_box)


def smooth(g, seed):
    """The workload field of dimension d (seeded), at the oracle's node coordinates."""
    return inputs.workload_field(g.d, g.coords(), seed)


OPS = [(1, 3, 3), (1, 16, 7), (1, 1, 4), (1, 5, 15), (2, 1, 3), (2, 2, 2), (2, 3, 4), (2, 5, 7),
       (2, 3, 15), (3, 1, 4), (3, 2, 2), (3, 3, 3), (3, 3, 7), (3, 2, 11), (3, 2, 12), (3, 1, 15), (3, 2, 13),
       (3, 2, 15)]


@pytest.mark.parametrize("dim,E,N", OPS)
def test_operators_match_oracle_fp64(dim, E, N):
    s, g = pair(dim, E, N)
    u, w = inputs.field_random(dim, g.G, 10 + N), inputs.field_random(dim, g.G, 20 + N)
    assert relerr(s.rhs(u), g.rhs(u)) < RTOL64
    assert relerr(s.jac(u, w), g.jac(u, w)) < RTOL64
    assert relerr(s.jacT(u, w), g.jacT(u, w)) < RTOL64


# FP32-bulk form, at the viscosities of the workloads (1D 1e-2, 2D 1e-3, 3D 5e-4).
# Its error is set by the cancellation, in the gather-scatter sum, of the large
# inter-element viscous flux terms of the lumped-mass weak form: about
# eps32 * nu (2/h)^2 / w_0 * h |grad u| / |F|, which stays below 1e-5 in this regime.
FP32_NU = {1: 1e-2, 2: 1e-3, 3: 5e-4}


@pytest.mark.parametrize("dim,E,N", [(1, 16, 7), (2, 16, 7), (2, 8, 9), (3, 6, 7), (3, 3, 15)])
def test_operators_match_oracle_fp32_bulk(dim, E, N):
    s, g = pair(dim, E, N, nu=FP32_NU[dim], precision="fp32_bulk")
    u, w = smooth(g, 1), smooth(g, 2)
    errs = {"F": relerr(s.rhs(u), g.rhs(u)), "J": relerr(s.jac(u, w), g.jac(u, w)),
            "JT": relerr(s.jacT(u, w), g.jacT(u, w))}
    assert max(errs.values()) < RTOL32, errs


# Every 3D FP32 element-pass layout: two partial tiles (n = 4, 5), one partial tile for F and
# J^T (n = 6..8), one for F only (n = 9..11), the shared pass code (n = 12) and the lean kernels
# (n = 13..16).
@pytest.mark.parametrize("E,N", [(3, 3), (3, 4), (3, 5), (2, 6), (2, 8), (2, 9), (2, 10), (2, 11), (2, 12), (2, 14)])
def test_fp32_bulk_3d_operators_at_every_pass_layout(E, N):
    s, g = pair(3, E, N, nu=FP32_NU[3], precision="fp32_bulk")
    u, w = smooth(g, 1), smooth(g, 2)
    errs = {"F": relerr(s.rhs(u), g.rhs(u)), "J": relerr(s.jac(u, w), g.jac(u, w)),
            "JT": relerr(s.jacT(u, w), g.jacT(u, w))}
    assert max(errs.values()) < RTOL32, errs


@pytest.mark.parametrize("dim,E,N,scheme,steps,dt", [(2, 8, 7, "ssprk3", 20, 2e-4), (3, 4, 7, "rk4", 8, 2.5e-4),
                                                    (1, 16, 7, "rk4", 50, 1e-3)])
def test_fp32_bulk_gradient_matches_fp64_oracle(dim, E, N, scheme, steps, dt):
    s, g = pair(dim, E, N, nu=FP32_NU[dim], precision="fp32_bulk")
    u0, uo = smooth(g, 1), smooth(g, 2)
    Jr, lam_ref, uN_ref = ork.objective_and_gradient(g, u0, uo, dt, steps, scheme)
    assert relerr(s.rk_forward(u0, dt, steps, scheme), uN_ref) < RTOL32
    J, grad = s.objective_grad(u0, uo, dt, steps, scheme)
    assert abs(J - Jr) <= RTOL32 * abs(Jr)
    assert relerr(grad, lam_ref) < RTOL32


def test_fp32_bulk_storage_modes_give_bitwise_equal_gradients():
    ref = None
    for mode, slots in (("stages", 0), ("states", 0), ("binomial", 3)):
        s, g = pair(2, 6, 7, nu=1e-3, precision="fp32_bulk", ckpt=mode, ckpt_slots=slots)
        J, grad = s.objective_grad(smooth(g, 1), smooth(g, 2), 2e-4, 15, "ssprk3")
        if ref is None:
            ref = (J, grad.clone())
        else:
            assert J == ref[0] and torch.equal(grad, ref[1])


@pytest.mark.parametrize("dim,E,N", [(1, 16, 7), (2, 8, 7), (3, 4, 7)])
def test_dot_product_identity_on_gpu(dim, E, N):
    s, g = pair(dim, E, N, nu=0.01)
    u, w, v = (torch.from_numpy(inputs.field_random(dim, g.G, k)).cuda() for k in (1, 2, 3))
    Jw, JTv = s.jac(u, w), s.jacT(u, v)
    lhs, rhs = float((Jw * v).sum()), float((w * JTv).sum())
    assert abs(lhs - rhs) <= 1e-12 * float(Jw.norm()) * float(v.norm())


def test_gather_scatter_is_bitwise_reproducible():
    s, g = pair(3, 4, 7)
    u, v = (torch.from_numpy(inputs.field_random(3, g.G, k)).cuda() for k in (5, 6))
    a1, b1 = s.rhs(u).clone(), s.jacT(u, v).clone()
    a2, b2 = s.rhs(u), s.jacT(u, v)
    assert torch.equal(a1, a2) and torch.equal(b1, b2)


@pytest.mark.parametrize("dim,E,N,scheme,steps,dt", [(1, 16, 7, "rk4", 40, 1e-3), (2, 4, 7, "ssprk3", 12, 2e-4),
                                                    (3, 3, 5, "rk4", 5, 5e-4), (2, 3, 4, "euler", 10, 1e-4)])
def test_rk_forward_matches_oracle(dim, E, N, scheme, steps, dt):
    s, g = pair(dim, E, N, nu=0.01)
    u0 = smooth(g, 1)
    ref, _ = ork.rk_forward(g.rhs, u0, dt, steps, scheme)
    assert relerr(s.rk_forward(u0, dt, steps, scheme), ref) < RTOL64


@pytest.mark.parametrize("mode,slots", [("stages", 0), ("states", 0), ("binomial", 1), ("binomial", 2),
                                        ("binomial", 3), ("binomial", 5)])
def test_adjoint_sweep_matches_oracle_in_every_storage_mode(mode, slots):
    dim, E, N, steps, dt, scheme = 2, 3, 5, 13, 3e-4, "rk4"
    s, g = pair(dim, E, N, nu=0.02, ckpt=mode, ckpt_slots=slots)
    u0, uo = smooth(g, 1), smooth(g, 2)
    Jr, lam_ref, _ = ork.objective_and_gradient(g, u0, uo, dt, steps, scheme)
    J, grad = s.objective_grad(u0, uo, dt, steps, scheme)
    assert abs(J - Jr) <= RTOL64 * abs(Jr)
    assert relerr(grad, lam_ref) < RTOL64
    st = s.sweep_stats()
    assert st["adjoint_jacT"] == 4 * steps
    if mode == "stages":
        assert st["adjoint_rhs"] == 0
    if mode == "states":
        assert st["adjoint_rhs"] == 3 * steps   # taping: s-1 stages per step


def test_binomial_gradient_is_bitwise_equal_to_store_all():
    dim, E, N, steps, dt = 2, 3, 4, 17, 2e-4
    ref = None
    for mode, slots in (("stages", 0), ("binomial", 1), ("binomial", 3), ("binomial", 4)):
        s, g = pair(dim, E, N, nu=0.02, ckpt=mode, ckpt_slots=slots)
        J, grad = s.objective_grad(smooth(g, 1), smooth(g, 2), dt, steps, "ssprk3")
        if ref is None:
            ref = (J, grad.clone())
        else:
            assert J == ref[0] and torch.equal(grad, ref[1])


def test_checkpointed_oracle_agrees_with_gpu_binomial():
    dim, E, N, steps, dt = 1, 8, 5, 20, 1e-3
    s, g = pair(dim, E, N, nu=0.02, ckpt="binomial", ckpt_slots=3)
    u0, lamT = smooth(g, 1), smooth(g, 2)
    uT = s.rk_forward(u0, dt, steps, "rk4")
    lam0 = s.rk_adjoint(torch.from_numpy(lamT).cuda())
    ref, count = checkpointed_gradient_lam0(g.rhs, g.jacT, u0, lamT, dt, steps, "rk4", 2)
    assert relerr(lam0, ref) < RTOL64
    assert relerr(uT, ork.rk_forward(g.rhs, u0, dt, steps, "rk4")[0]) < RTOL64


def test_objective_matches_oracle():
    s, g = pair(3, 3, 4)
    u, uo = inputs.field_random(3, g.G, 1), inputs.field_random(3, g.G, 2)
    lam = s.empty()
    J = s.objective(u, uo, lam)
    Jr, lr = g.objective(u, uo)
    assert abs(J - Jr) <= 1e-13 * abs(Jr)
    assert relerr(lam, lr) < 1e-14


def test_gradient_taylor_remainder_on_gpu():
    s, g = pair(2, 6, 7, nu=0.01)
    u0, uo = torch.from_numpy(smooth(g, 1)).cuda(), torch.from_numpy(smooth(g, 2)).cuda()
    du = torch.from_numpy(inputs.field_random(2, g.G, 9)).cuda() * 0.1
    J0, grad = s.objective_grad(u0, uo, 2e-4, 20, "ssprk3")
    slope = float((grad * du).sum())
    rem = []
    for eps in (1e-1, 1e-2, 1e-3):
        J1, _ = s.objective_grad(u0 + eps * du, uo, 2e-4, 20, "ssprk3")
        rem.append(abs(J1 - J0 - eps * slope))
    assert rem[1] < rem[0] / 50 and rem[2] < rem[1] / 50


def test_autograd_function_gradient():
    s, g = pair(2, 4, 5, nu=0.01)
    u0 = torch.from_numpy(smooth(g, 1)).cuda().requires_grad_(True)
    uo = torch.from_numpy(smooth(g, 2)).cuda()
    J = SemMisfit.apply(u0, s, uo, 2e-4, 10, "rk4")
    J.backward()
    Jr, lam_ref, _ = ork.objective_and_gradient(g, smooth(g, 1), smooth(g, 2), 2e-4, 10, "rk4")
    assert abs(float(J) - Jr) <= RTOL64 * abs(Jr)
    assert relerr(u0.grad, lam_ref) < RTOL64


def test_autograd_function_forward_runs_no_adjoint_and_survives_an_intervening_forward():
    s, g = pair(2, 4, 5, nu=0.01)
    u0a = torch.from_numpy(smooth(g, 1)).cuda().requires_grad_(True)
    u0b = torch.from_numpy(smooth(g, 3)).cuda().requires_grad_(True)
    uo = torch.from_numpy(smooth(g, 2)).cuda()
    Ja = SemMisfit.apply(u0a, s, uo, 2e-4, 10, "rk4")
    torch.cuda.synchronize()
    assert s.sweep_stats()["adjoint_jacT"] == 0          # forward only: no adjoint sweep yet
    Jb = SemMisfit.apply(u0b, s, uo, 2e-4, 10, "rk4")   # overwrites the handle's trajectory
    Ja.backward()
    Jref, gref = s.objective_grad(u0a.detach(), uo, 2e-4, 10, "rk4")
    assert float(Ja) == Jref
    assert torch.equal(u0a.grad, gref)
    Jb.backward()
    _, gref_b = s.objective_grad(u0b.detach(), uo, 2e-4, 10, "rk4")
    assert torch.equal(u0b.grad, gref_b)


def test_host_buffers_give_the_same_result():
    s, g = pair(2, 4, 7)
    u0 = torch.from_numpy(smooth(g, 1)).pin_memory()
    uo = torch.from_numpy(smooth(g, 2)).pin_memory()
    J1, g1 = s.objective_grad(u0, uo, 2e-4, 5, "ssprk3", host=True)
    J2, g2 = s.objective_grad(u0.cuda(), uo.cuda(), 2e-4, 5, "ssprk3")
    assert J1 == J2 and torch.equal(g1, g2.cpu())


def test_error_codes_on_gpu():
    s, g = pair(2, 3, 4)
    u = torch.from_numpy(inputs.field_random(2, g.G, 1)).cuda()
    bad = u.clone()
    bad[0, 1, 1] = float("nan")
    with pytest.raises(L.SemError) as ei:
        s.rk_forward(bad, 1e-4, 3, "rk4")
    assert ei.value.code == L.SEM_ERR_NONFINITE
    with pytest.raises(L.SemError) as ei:
        s.rhs(u, out=u)
    assert ei.value.code == L.SEM_ERR_ALIAS
    s2 = Sem(2, 3, 4, 0.01, ckpt="stages", ckpt_budget_bytes=1024)
    with pytest.raises(L.SemError) as ei:
        s2.rk_forward(u, 1e-4, 3, "rk4")
    assert ei.value.code == L.SEM_ERR_OOM
    s3 = Sem(2, 3, 4, 0.01)
    with pytest.raises(L.SemError) as ei:
        s3.rk_adjoint(u)
    assert ei.value.code == L.SEM_ERR_STATE


# ------------------------------------------------------------ full workload sizes
def test_full_size_2d_operators_match_oracle():
    """2D vector Burgers, E = 64^2 quads, N = 7 (401,408 unknowns): every output compared."""
    s, g = pair(2, 64, 7, nu=1e-3)
    u, v = smooth(g, 1), smooth(g, 2)
    assert relerr(s.rhs(u), g.rhs(u)) < RTOL64
    assert relerr(s.jacT(u, v), g.jacT(u, v)) < RTOL64


def test_full_size_2d_gradient_short_horizon_matches_oracle():
    """Same grid, SSP-RK3 with dt = 2e-4: 8 steps of the gradient evaluation, all outputs compared."""
    s, g = pair(2, 64, 7, nu=1e-3)
    u0, uo = smooth(g, 1), smooth(g, 2)
    Jr, lam_ref, _ = ork.objective_and_gradient(g, u0, uo, 2e-4, 8, "ssprk3")
    J, grad = s.objective_grad(u0, uo, 2e-4, 8, "ssprk3")
    assert abs(J - Jr) <= RTOL64 * abs(Jr)
    assert relerr(grad, lam_ref) < RTOL64


def _sample_nodes(g, rng, k):
    nodes = [tuple(int(x) for x in rng.integers(0, g.G, g.d)) for _ in range(k)]
    # element corners, edges and faces (shared by 8, 4, 2 elements) and the periodic seam
    N, G = g.N, g.G
    nodes += [(0, 0, 0), (N, 2 * N, G - N), (0, 3, 5), (N, N + 1, 1), (G - 1, G - 1, G - 1), (1, 0, 2 * N)]
    return nodes


@pytest.mark.parametrize("prec,rtol", [("fp64", RTOL64), ("fp32_bulk", RTOL32)])
def test_full_size_3d_operators_on_sampled_nodes(prec, rtol):
    """3D vector Burgers, E = 32^3 hexes, N = 7 (33.7M unknowns): sampled outputs vs the oracle."""
    s, g = pair(3, 32, 7, nu=5e-4, precision=prec)
    x = g.coords()
    u, v = inputs.field_3d(x, 1), inputs.field_3d(x, 2)
    F, JT = s.rhs(u).cpu().numpy(), s.jacT(u, v).cpu().numpy()
    nodes = _sample_nodes(g, np.random.default_rng(0), 40)
    Fr, JTr = g.rhs_at(u, nodes), g.jacT_at(u, v, nodes)
    scaleF = np.max(np.abs(Fr))
    scaleT = np.max(np.abs(JTr))
    for k, nd in enumerate(nodes):
        for c in range(3):
            assert abs(F[(c,) + nd] - Fr[c, k]) <= rtol * scaleF
            assert abs(JT[(c,) + nd] - JTr[c, k]) <= rtol * scaleT


def test_fp32_rows_of_more_than_32_elements_on_sampled_nodes():
    """E = 36 hexes per side, N = 7 (3 x 252^3 unknowns): the row-wise FP32 assembly covers each
    grid row in two warp chunks (32 elements, then a ragged 4), with the periodic seam between the
    last chunk and the first.  F and J^T on sampled nodes against the oracle."""
    s, g = pair(3, 36, 7, nu=5e-4, precision="fp32_bulk")
    x = g.coords()
    u, v = inputs.field_3d(x, 1), inputs.field_3d(x, 2)
    F, JT = s.rhs(u).cpu().numpy(), s.jacT(u, v).cpu().numpy()
    N, G = g.N, g.G
    nodes = _sample_nodes(g, np.random.default_rng(5), 24)
    # nodes in the second chunk of a row (elements 32..35 along x) and at the seam
    nodes += [(3, 5, 32 * N), (N, 0, 33 * N + 2), (0, 2 * N, G - 1), (7, 9, 31 * N + 6), (4, 4, 0)]
    Fr, JTr = g.rhs_at(u, nodes), g.jacT_at(u, v, nodes)
    sF, sT = np.max(np.abs(Fr)), np.max(np.abs(JTr))
    for k, nd in enumerate(nodes):
        for c in range(3):
            assert abs(F[(c,) + nd] - Fr[c, k]) <= RTOL32 * sF
            assert abs(JT[(c,) + nd] - JTr[c, k]) <= RTOL32 * sT


@pytest.mark.parametrize("mode,slots", [("stages", 0), ("binomial", 3)])
def test_graph_replay_equals_stream_launches(mode, slots):
    s, g = pair(2, 6, 7, nu=1e-3, ckpt=mode, ckpt_slots=slots)
    u0, uo = torch.from_numpy(smooth(g, 1)).cuda(), torch.from_numpy(smooth(g, 2)).cuda()
    J0, g0 = s.objective_grad(u0, uo, 2e-4, 9, "ssprk3")
    g0 = g0.clone()
    s.use_graph(True)
    grad = s.empty()
    for _ in range(3):
        J1, g1 = s.objective_grad(u0, uo, 2e-4, 9, "ssprk3", grad=grad)
        assert J1 == J0 and torch.equal(g1, g0)
    assert s.graph_replays() == 3


def test_kernel_timing_inside_a_replayed_graph():
    s, g = pair(2, 6, 7, nu=1e-3)
    u0, uo = torch.from_numpy(smooth(g, 1)).cuda(), torch.from_numpy(smooth(g, 2)).cuda()
    s.profile(4)
    s.use_graph(True)
    s.objective_grad(u0, uo, 2e-4, 8, "ssprk3")        # records the graph, then replays it
    first = s.profile_read(reset=True)
    s.objective_grad(u0, uo, 2e-4, 8, "ssprk3")        # replay only
    second = s.profile_read(reset=True)
    # 8 steps x 3 stages of F and of J^T, one in 4 of each kind timed, every replay
    assert second["rhs"][1] == 6 and second["jacT"][1] == 6 and second["assemble"][1] == 12
    assert first["rhs"][1] == second["rhs"][1]
    assert all(second[k][0] > 0 for k in ("rhs", "jacT", "assemble"))
    # every timed assembly reads the element-local values and writes at least one output
    d, E, N = 2, 6, 7
    lvec, ndof = d * (E * (N + 1)) ** d * 8, d * (E * N) ** d
    assert lvec + ndof * 8 <= second["assemble"][2] / 12 <= lvec + 7 * ndof * 8


@pytest.mark.parametrize("prec,lw", [("fp64", 8), ("fp32_bulk", 4)])
@pytest.mark.parametrize("dim,E,N", [(2, 6, 7), (3, 3, 5)])
def test_assembly_bytes_of_timed_applies(dim, E, N, prec, lw):
    """The library counts the algorithmic bytes of each timed assembly: the element-local values
    once, plus 8 bytes per unknown for each epilogue source and output."""
    s, g = pair(dim, E, N, precision=prec)
    u = torch.from_numpy(smooth(g, 1)).cuda()
    s.profile(1)
    s.rhs(u)
    s.jacT(u, u)
    p = s.profile_read(reset=True)
    lvec, ndof = dim * (E * (N + 1)) ** dim * lw, dim * (E * N) ** dim
    assert p["assemble"][1] == 2 and p["assemble"][2] == 2 * (lvec + ndof * 8)
    assert p["rhs"][1] == 1 and p["rhs"][2] == 0 and p["jacT"][1] == 1
    s.profile(0)


# Degenerate cases: the lowest order (two points per direction), no viscosity, the zero field.
@pytest.mark.parametrize("prec", ["fp64", "fp64_df"])
@pytest.mark.parametrize("dim,E,N", [(1, 4, 1), (2, 3, 1), (3, 2, 1), (2, 5, 2)])
def test_lowest_orders_match_oracle(dim, E, N, prec):
    s, g = Sem(dim, E, N, 0.037, precision=prec), Grid(dim, E, N, 0.037)
    u, w = inputs.field_random(dim, g.G, 30 + dim), inputs.field_random(dim, g.G, 40 + dim)
    assert relerr(s.rhs(u), g.rhs(u)) < RTOL64
    assert relerr(s.jac(u, w), g.jac(u, w)) < RTOL64
    assert relerr(s.jacT(u, w), g.jacT(u, w)) < RTOL64


@pytest.mark.parametrize("prec", ["fp64", "fp64_df", "fp32_bulk"])
def test_inviscid_and_zero_fields(prec):
    s, g = Sem(2, 4, 5, 0.0, precision=prec), Grid(2, 4, 5, 0.0)
    u, w = smooth(g, 1), smooth(g, 2)
    tol = RTOL32 if prec == "fp32_bulk" else RTOL64
    assert relerr(s.rhs(u), g.rhs(u)) < tol
    assert relerr(s.jacT(u, w), g.jacT(u, w)) < tol
    z = np.zeros_like(u)
    assert float(s.rhs(z).abs().max()) == 0.0          # F(0) = 0 exactly
    assert float(s.jacT(z, z).abs().max()) == 0.0


def test_dependent_launch_changes_no_result():
    """Programmatic dependent launch only overlaps launch latency: the same bits either way."""
    try:
        out = []
        for on in (1, 0):
            L.lib().sem_set_dependent_launch(on)
            s = Sem(2, 6, 7, 1e-3)
            s.use_graph(True)
            x = s.coords()
            u0, uo = inputs.workload_field(2, x, 1), inputs.workload_field(2, x, 2)
            J, g = s.objective_grad(u0, uo, 2e-4, 10, "ssprk3")
            out.append((J, g.clone(), s.rhs(u0).clone()))
        assert out[0][0] == out[1][0] and torch.equal(out[0][1], out[1][1]) and torch.equal(out[0][2], out[1][2])
    finally:
        L.lib().sem_set_dependent_launch(1)
