"""Python front end of libsem over torch tensors (device memory and streams only).

Every operation is one call into the C ABI; torch supplies the CUDA buffers and
the current stream.  Inputs may be CPU tensors or numpy arrays for the
end-to-end form: they are copied to the device (pinned host memory when given)
and results copied back, which is the host-buffer path the benchmarks time.
"""
import ctypes

import numpy as np
import torch

from . import _lib as L

SCHEMES = {"rk4": L.SEM_RK4, "ssprk3": L.SEM_SSPRK3, "euler": L.SEM_EULER, "cn": L.SEM_CN, "bs3": L.SEM_BS3}
PRECISIONS = {"fp64": L.SEM_PREC_FP64, "fp32_bulk": L.SEM_PREC_FP32_BULK, "fp64_df": L.SEM_PREC_FP64_DF}
CKPT = {"auto": L.SEM_CKPT_AUTO, "stages": L.SEM_CKPT_STAGES, "states": L.SEM_CKPT_STATES,
        "binomial": L.SEM_CKPT_BINOMIAL, "two_level": L.SEM_CKPT_TWO_LEVEL}


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _device(device):
    """The handle's device with an explicit index (a bare "cuda" means the current device)."""
    if device is None:
        return torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() \
            else torch.device("cpu")
    device = torch.device(device)
    if device.type == "cuda" and device.index is None:
        device = torch.device("cuda", torch.cuda.current_device())
    return device


class Sem:
    """Periodic d-dimensional viscous Burgers on E^d GLL elements of order N (one GPU)."""

    _fwd_token = 0     # counts forward sweeps run through this object (the handle keeps the last trajectory)

    def __init__(self, dim, E, N, nu, L_box=None, precision="fp64", ckpt="auto", ckpt_slots=0,
                 ckpt_budget_bytes=0, device=None):
        o = L.sem_opts(dim=dim, E=E, N=N, nu=float(nu), L=float(L_box or 0.0),
                       precision=PRECISIONS[precision], ckpt_mode=CKPT[ckpt], ckpt_slots=ckpt_slots,
                       ckpt_budget_bytes=ckpt_budget_bytes)
        h = ctypes.c_void_p()
        L.check(L.lib().sem_create_ex(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.dim, self.E, self.N, self.nu = dim, E, N, float(nu)
        self.G = E * N
        self.ndof = int(L.lib().sem_ndof(h))
        self.shape = (dim,) + (self.G,) * dim
        self.device = _device(device)

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_h", None):
            L.lib().sem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ helpers
    def coords(self):
        x = np.empty(self.G)
        L.check(L.lib().sem_coords(self._h, x.ctypes.data_as(ctypes.c_void_p)))
        return x

    def empty(self):
        return torch.empty(self.shape, dtype=torch.float64, device=self.device)

    def _dev(self, t, name):
        if isinstance(t, np.ndarray):
            t = torch.from_numpy(np.ascontiguousarray(t, dtype=np.float64))
        if not isinstance(t, torch.Tensor):
            raise TypeError("%s must be a tensor or ndarray" % name)
        if t.dtype != torch.float64:
            raise TypeError("%s must be float64" % name)
        if t.numel() != self.ndof:
            raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), self.ndof))
        if t.device != self.device:
            t = t.to(self.device, non_blocking=t.is_pinned())
        return t.contiguous().view(self.shape)

    def _out(self, t, name):
        """A caller's output buffer, written in place by the library: it must already be a
        contiguous float64 tensor of ndof values on the handle's device (None: a new one)."""
        if t is None:
            return self.empty()
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64:
            raise TypeError("%s must be a float64 tensor" % name)
        if t.device != self.device:
            raise ValueError("%s is on %s, the handle on %s" % (name, t.device, self.device))
        if t.numel() != self.ndof or not t.is_contiguous():
            raise ValueError("%s must be contiguous with %d elements" % (name, self.ndof))
        return t

    @staticmethod
    def _p(t):
        return ctypes.c_void_p(t.data_ptr())

    # ------------------------------------------------------------ operators
    def rhs(self, u, out=None):
        u = self._dev(u, "u")
        out = self._out(out, "out")
        L.check(L.lib().sem_rhs(self._h, self._p(u), self._p(out), _stream(self.device)))
        return out

    def jac(self, u, w, out=None):
        u, w = self._dev(u, "u"), self._dev(w, "w")
        out = self._out(out, "out")
        L.check(L.lib().sem_jac_apply(self._h, self._p(u), self._p(w), self._p(out), _stream(self.device)))
        return out

    def jacT(self, u, v, out=None):
        u, v = self._dev(u, "u"), self._dev(v, "v")
        out = self._out(out, "out")
        L.check(L.lib().sem_jacT_apply(self._h, self._p(u), self._p(v), self._p(out), _stream(self.device)))
        return out

    # ------------------------------------------------------------ sweeps
    def rk_forward(self, u0, dt, nsteps, scheme="rk4", out=None):
        u0 = self._dev(u0, "u0")
        out = self._out(out, "out")
        self._fwd_token += 1           # the handle now keeps this sweep's trajectory
        L.check(L.lib().sem_rk_forward(self._h, SCHEMES[scheme], float(dt), int(nsteps), self._p(u0),
                                       self._p(out), _stream(self.device)))
        return out

    def rk_adjoint(self, lamT, out=None):
        lamT = self._dev(lamT, "lamT")
        out = self._out(out, "out")
        L.check(L.lib().sem_rk_adjoint(self._h, self._p(lamT), self._p(out), _stream(self.device)))
        return out

    def objective(self, u, u_obs, lam=None):
        u, u_obs = self._dev(u, "u"), self._dev(u_obs, "u_obs")
        lam = self._out(lam, "lam") if lam is not None else None
        J = ctypes.c_double()
        L.check(L.lib().sem_objective(self._h, self._p(u), self._p(u_obs), ctypes.byref(J),
                                      self._p(lam) if lam is not None else None, _stream(self.device)))
        return J.value

    def objective_grad(self, u0, u_obs, dt, nsteps, scheme="rk4", grad=None, host=False):
        """(J, dJ/du0).  With host=True the gradient is returned as a CPU tensor."""
        u0, u_obs = self._dev(u0, "u0"), self._dev(u_obs, "u_obs")
        grad = self._out(grad, "grad")
        J = ctypes.c_double()
        self._fwd_token += 1
        L.check(L.lib().sem_objective_grad(self._h, SCHEMES[scheme], float(dt), int(nsteps), self._p(u0),
                                           self._p(u_obs), ctypes.byref(J), self._p(grad),
                                           _stream(self.device)))
        return J.value, (grad.cpu() if host else grad)

    def set_contraction(self, mode="cuda_core"):
        """Contraction engine of the element kernels: "cuda_core" (even-odd FMA chains, default) or
        "tensor" (3D, N = 15: tcgen05 split-TF32 in the FP32-bulk form, DMMA in FP64; F only)."""
        m = {"cuda_core": L.SEM_CONTRACT_CUDA_CORE, "tensor": L.SEM_CONTRACT_TENSOR}[mode]
        L.check(L.lib().sem_set_contraction(self._h, m))

    def use_graph(self, enable=True):
        """Record the gradient evaluation as a CUDA graph once and replay it (sem_set_graph)."""
        L.check(L.lib().sem_set_graph(self._h, 1 if enable else 0))

    def graph_replays(self):
        return int(L.lib().sem_graph_replays(self._h))

    def profile(self, every=1):
        """Time one launch in `every` per kernel kind (0: off)."""
        L.check(L.lib().sem_profile(self._h, int(every)))

    def profile_read(self, reset=True):
        """{kind: (ms, timed launches, algorithmic bytes)} for kinds rhs, jac, jacT element kernels
        and assembly (bytes are counted for the assembly only)."""
        ms = (ctypes.c_double * 4)()
        n = (ctypes.c_longlong * 4)()
        nb = (ctypes.c_double * 4)()
        L.check(L.lib().sem_profile_read(self._h, ms, n, nb, 1 if reset else 0))
        return {k: (ms[i], n[i], nb[i]) for i, k in enumerate(("rhs", "jac", "jacT", "assemble"))}

    def sweep_stats(self):
        out = (ctypes.c_longlong * 3)()
        L.check(L.lib().sem_sweep_stats(self._h, out))
        return {"forward_rhs": out[0], "adjoint_rhs": out[1], "adjoint_jacT": out[2]}

    def set_advection(self, a=None):
        """Integrate du/dt = J(a) u (frozen advecting field a) instead of Burgers; None: back to Burgers."""
        if a is None:
            L.check(L.lib().sem_set_advection(self._h, None, _stream(self.device)))
            self._frozen = None
            return
        a = self._dev(a, "a")
        L.check(L.lib().sem_set_advection(self._h, self._p(a), _stream(self.device)))
        self._frozen = a   # kept alive until the copy on the stream has run

    def launch_count(self):
        """Element and assembly launches since the last forward sweep began (sem_launch_count)."""
        n = ctypes.c_longlong()
        L.check(L.lib().sem_launch_count(self._h, ctypes.byref(n)))
        return n.value

    def set_adaptive(self, atol=0.0, rtol=0.0):
        """Adaptive steps for scheme "bs3" (sem_set_adaptive); dt * nsteps is then the horizon."""
        L.check(L.lib().sem_set_adaptive(self._h, float(atol), float(rtol)))

    def adaptive_steps(self):
        """(accepted step sizes as an ndarray, rejected count) of the last adaptive sweep."""
        acc, rej = ctypes.c_int(), ctypes.c_int()
        L.check(L.lib().sem_adaptive_steps(self._h, ctypes.byref(acc), ctypes.byref(rej), None, 0))
        dts = np.empty(acc.value)
        L.check(L.lib().sem_adaptive_steps(self._h, ctypes.byref(acc), ctypes.byref(rej),
                                           dts.ctypes.data_as(ctypes.c_void_p), int(dts.size)))
        return dts, rej.value

    def set_host_tier(self, host_bytes):
        """Pinned host memory for the second level of the trajectory store (sem_set_host_tier)."""
        L.check(L.lib().sem_set_host_tier(self._h, int(host_bytes)))

    def trajectory_info(self):
        out = (ctypes.c_longlong * 4)()
        L.check(L.lib().sem_trajectory_info(self._h, out))
        modes = {v: k for k, v in CKPT.items()}
        return {"mode": modes.get(out[0], None) if out[0] else None, "device": out[1], "host": out[2],
                "slots": out[3]}

    def set_solver(self, newton_rtol=1e-12, krylov_rtol=1e-12, krylov_m=30, krylov_maxit=2000):
        """Newton / GMRES settings of the Crank-Nicolson scheme (sem_set_solver)."""
        L.check(L.lib().sem_set_solver(self._h, float(newton_rtol), float(krylov_rtol), int(krylov_m),
                                       int(krylov_maxit)))

    def solver_stats(self):
        out = (ctypes.c_longlong * 4)()
        L.check(L.lib().sem_solver_stats(self._h, out))
        return {"newton": out[0], "forward_krylov": out[1], "adjoint_krylov": out[2], "applies": out[3]}


class SemBatch(Sem):
    """Independent 2D instances (E[k], N[k], nu[k]) on packed vectors (sem_batch_create).

    Every Sem operation works on packed tensors of `ndof` values; `pack` and
    `unpack` convert between per-instance (2, G_k, G_k) arrays and the packed form.
    """

    def __init__(self, E, N, nu, L_box=None, ckpt="auto", ckpt_slots=0, ckpt_budget_bytes=0, device=None):
        count = len(E)
        o = L.sem_opts(dim=2, E=0, N=0, nu=0.0, L=float(L_box or 0.0), precision=L.SEM_PREC_FP64,
                       ckpt_mode=CKPT[ckpt], ckpt_slots=ckpt_slots, ckpt_budget_bytes=ckpt_budget_bytes)
        Ea = (ctypes.c_int * count)(*[int(e) for e in E])
        Na = (ctypes.c_int * count)(*[int(n) for n in N])
        nua = (ctypes.c_double * count)(*[float(v) for v in nu])
        h = ctypes.c_void_p()
        L.check(L.lib().sem_batch_create(count, Ea, Na, nua, ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self.dim, self.count = 2, count
        self.E, self.N, self.nu = list(E), list(N), list(nu)
        self.ndof = int(L.lib().sem_ndof(h))
        self.shape = (self.ndof,)
        self.layout = []
        for k in range(count):
            off, n = ctypes.c_size_t(), ctypes.c_size_t()
            L.check(L.lib().sem_batch_layout(h, k, ctypes.byref(off), ctypes.byref(n)))
            self.layout.append((off.value, n.value))
        self.device = _device(device)

    def coords(self, k):
        x = np.empty(self.E[k] * self.N[k])
        L.check(L.lib().sem_batch_coords(self._h, int(k), x.ctypes.data_as(ctypes.c_void_p)))
        return x

    def pack(self, fields):
        """Concatenate per-instance (2, G_k, G_k) arrays into one packed float64 array."""
        return np.concatenate([np.ascontiguousarray(f, dtype=np.float64).ravel() for f in fields])

    def unpack(self, packed):
        out = []
        for k, (off, n) in enumerate(self.layout):
            G = self.E[k] * self.N[k]
            out.append(packed[off:off + n].reshape(2, G, G))
        return out

    def autotune(self):
        ms = (ctypes.c_double * 4)()
        th = ctypes.c_int()
        L.check(L.lib().sem_batch_autotune(self._h, ms, ctypes.byref(th), _stream(self.device)))
        return th.value, list(ms)

    def objective_grad_each(self, u0, u_obs, dt, nsteps, scheme="rk4", grad=None):
        """(per-instance misfits, packed gradient)."""
        u0, u_obs = self._dev(u0, "u0"), self._dev(u_obs, "u_obs")
        grad = self._out(grad, "grad")
        J = (ctypes.c_double * self.count)()
        L.check(L.lib().sem_batch_objective_grad(self._h, SCHEMES[scheme], float(dt), int(nsteps), self._p(u0),
                                                 self._p(u_obs), J, self._p(grad), _stream(self.device)))
        return list(J), grad


def ckpt_plan(nsteps, slots):
    """Optimal advance count of the binomial schedule (host only)."""
    a = ctypes.c_longlong()
    L.check(L.lib().sem_ckpt_plan(int(nsteps), int(slots), ctypes.byref(a)))
    return a.value


class SemMisfit(torch.autograd.Function):
    """u0 -> J(u0) = 1/2 ||u_N(u0) - u_obs||_M^2 with backward = the discrete adjoint sweep.

    forward runs the forward sweep (sem_rk_forward, which keeps the trajectory
    the adjoint needs) and the misfit with its terminal adjoint M (u_N - u_obs);
    backward runs the adjoint sweep (sem_rk_adjoint) from that terminal adjoint
    and scales the gradient by the incoming gradient.  A forward-only use pays no
    adjoint sweep.  If another forward sweep ran on the same handle in between
    (the handle keeps only the last trajectory), backward repeats this one first.
    """

    @staticmethod
    def forward(ctx, u0, sem, u_obs, dt, nsteps, scheme):
        u0d = u0.detach()
        uN = sem.rk_forward(u0d, dt, nsteps, scheme)
        lam = sem.empty()
        J = sem.objective(uN, u_obs, lam)
        ctx.sem, ctx.args, ctx.token = sem, (u0d, dt, nsteps, scheme), sem._fwd_token
        ctx.save_for_backward(lam)
        return torch.tensor(J, dtype=torch.float64, device=u0.device)

    @staticmethod
    def backward(ctx, gJ):
        (lam,) = ctx.saved_tensors
        sem = ctx.sem
        if sem._fwd_token != ctx.token:
            u0d, dt, nsteps, scheme = ctx.args
            sem.rk_forward(u0d, dt, nsteps, scheme)
        g = sem.rk_adjoint(lam)
        return gJ * g, None, None, None, None, None
