#!/usr/bin/env python
"""Throughput benchmark of the spectral-element Burgers gradient on GB300.

One step = one gradient evaluation of the misfit J(u0) = 1/2 ||u_N(u0) - u_obs||_M^2.
The default workload is the 3D vector viscous Burgers problem (periodic [0,1]^3,
32^3 hexahedra of order 7, 33,718,272 unknowns, nu = 5e-4, RK4 with dt = 2.5e-4,
binomial checkpointing with 20 slots) in FP64: forward sweep, misfit and terminal
adjoint, backward sweep with the matrix-free transpose Jacobian and the
checkpoint replays, all on one GPU through the C ABI.  The horizon is 300 steps:
past about 400 steps the seeded k^-5/3 field steepens into fronts the grid does
not resolve at this viscosity and the discrete solution diverges.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload 2d|3d|...]

N > 1 runs one independent replica per GPU (torchrun, one rank per GPU): the
path has no exchange step between GPUs, so scaling is weak.  Prints one JSON line.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GDOF/s for F(u) and J^T v; adjoint/forward cost ratio; gradient evals/s"

WORKLOADS = {
    "2d": dict(dim=2, E=64, N=7, nu=1e-3, scheme="ssprk3", dt=2e-4, nsteps=2000, ckpt="stages", slots=0,
               oracle_steps=10,
               desc="2D vector viscous Burgers, periodic [0,1]^2, 64x64 quads, N=7 (401,408 unknowns), "
                    "nu=1e-3, SSP-RK3 dt=2e-4 x 2000 steps, all stages stored; one gradient evaluation per step",
               data="synthetic: seeded 16-mode Fourier fields (|k|_inf <= 8, amplitude ~|k|^-2, max|u0| = 1) "
                    "for u0 (seed 1) and u_obs (seed 2)"),
    # the 3D horizons stop before the fields steepen past what the grid resolves: at these
    # viscosities the discrete solution (FP64 and FP32 alike) diverges near step 450 (N=7)
    # and step 350 (N=15)
    "3d": dict(dim=3, E=32, N=7, nu=5e-4, scheme="rk4", dt=2.5e-4, nsteps=300, ckpt="binomial", slots=20,
               oracle_steps=1,
               desc="3D vector viscous Burgers, periodic [0,1]^3, 32^3 hexes, N=7 (33,718,272 unknowns), "
                    "nu=5e-4, RK4 dt=2.5e-4 x 300 steps (T=0.075), binomial checkpointing with 20 slots",
               horizon="300 of the configured 1000 steps: the seeded k^-5/3 field steepens into fronts this grid "
                       "does not resolve at nu=5e-4, and the discrete solution (FP64 and FP32 alike) grows past "
                       "max|u| = 1.08 at step 400 and is non-finite by step 500; at step 300 max|u| <= 0.99",
               data="synthetic: seeded random-phase fields, spectrum ~k^-5/3 cut at |k| = 16, max|u0| = 1"),
    "batch": dict(dim=2, E=None, N=None, nu=1e-3, scheme="rk4", dt=1.5e-4, nsteps=300, ckpt="states", slots=0,
                  count=256,
                  desc="256 independent 2D vector viscous Burgers instances, periodic [0,1]^2, E per side drawn "
                       "from {8,16,24,32,48} and N from {5,7,9} (seed 4), nu=1e-3, RK4 dt=1.5e-4 x 300 steps, "
                       "one persistent launch per operator pass, every step's state stored (stages recomputed); one "
                       "batched gradient evaluation per step (256 instance gradients)",
                  data="synthetic: per instance k seeded 16-mode Fourier fields (seeds 1000+2k, 1001+2k)"),
    "3d15": dict(dim=3, E=16, N=15, nu=2e-4, scheme="rk4", dt=2e-4, nsteps=300, ckpt="states", slots=0,
                 oracle_steps=1,
                 desc="3D vector viscous Burgers, periodic [0,1]^3, 16^3 hexes, N=15 (41,472,000 unknowns), "
                      "nu=2e-4, RK4 dt=2e-4 x 300 steps (T=0.06), every step's state stored (stages recomputed)",
                 horizon="300 of the configured 400 steps: the discrete solution diverges between steps 340 and "
                         "360 at nu=2e-4 (the seeded field steepens past what the grid resolves)",
                 data="synthetic: seeded random-phase fields, spectrum ~k^-5/3 cut at |k| = 16, max|u0| = 1"),
    "2dcn": dict(dim=2, E=64, N=7, nu=1e-3, scheme="cn", dt=2e-3, nsteps=200, ckpt="states", slots=0,
                 desc="2D vector viscous Burgers, periodic [0,1]^2, 64x64 quads, N=7 (401,408 unknowns), "
                      "nu=1e-3, Crank-Nicolson dt=2e-3 x 200 steps (Newton + GMRES(30) to 1e-12 per step), "
                      "every state stored; one gradient evaluation per step",
                 data="synthetic: seeded 16-mode Fourier fields (|k|_inf <= 8, amplitude ~|k|^-2, max|u0| = 1) "
                      "for u0 (seed 1) and u_obs (seed 2)"),
    "1d": dict(dim=1, E=16, N=7, nu=0.01, scheme="rk4", dt=1e-3, nsteps=500, ckpt="stages", slots=0,
               oracle_steps=100,
               desc="1D viscous Burgers, periodic [0,2pi), 16 elements, N=7 (112 unknowns), nu=0.01, "
                    "RK4 dt=1e-3 x 500 steps",
               data="synthetic: u0 = sin x + 0.1 sum_k a_k sin(kx + phi_k), seeded"),
}

# FP64 FMA peak of one GB300: 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz
# (nominal 1.25 TFLOP/s; an FMA-chain probe measured 1.251 TFLOP/s).  FP32: 128
# FMA lanes per SM.
PEAK_FP64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# Double-float element arithmetic: a compensated multiply-add costs 13 FP32 operations.
PEAK_DF_TFLOPS = 152 * 128 * 2.07e9 / 13 * 2 / 1e12

# DRAM traffic per launch (bytes) of the dominant kernel from one ncu capture,
# valid only while the kernel sources hash to the recorded value.
TRAFFIC = {
    "rhs3_f64_kernel<8>@3d@fp64": {
        "bytes": int(round((181718016 + 218584832) * 32 ** 3 / 28 ** 3)), "src": "f76a8708d1d3acf3",
        "capture": "dram__bytes_read.sum + dram__bytes_write.sum of one rhs3_f64_kernel<8> launch at 28^3 hexes, "
                   "N=7 (ncu --set full), scaled to 32^3 hexes by the element count"},
    "jact2_kernel<double,8>@2d@fp64": {
        "bytes": 6477312 + 0, "src": "f76a8708d1d3acf3",
        "capture": "dram__bytes_read.sum + dram__bytes_write.sum of one jact2 launch at 64x64 quads, N=7 "
                   "(ncu --set full capture of the 2D FP64 element kernels)"},
    "op2c_kernel<semk::dfa::dfloat,8> (J^T)@2d@fp64_df": {
        "bytes": 6536192 + 0, "src": "f76a8708d1d3acf3",
        "capture": "dram__bytes_read.sum + dram__bytes_write.sum of one J^T launch (op2c_kernel) at 64x64 "
                   "quads, N=7 (ncu --set full capture of the 2D FP64-DF element kernels)"},
}

# sources of the element kernels (rhs*, jac*, jact*) and of the assembly kernels
KERNEL_SOURCES = {"elem": ["op_kernels.cuh", "op_elem.cuh", "op_elem_lean.cuh", "op_launch.cuh", "df64.cuh",
                           "op_d1.cu", "op_d2.cu", "op_d2_df.cu", "op_d3.cu", "op_d3_f.cu", "op_d3_df.cu",
                           "op_d3_df_mid.cu", "op_d3_df_hi.cu"],
                  "assemble": ["vec_kernels.cu", "asm_epi.cuh", "df64.cuh"]}


def kernel_src_hash(family):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[family]:
        with open(os.path.join(ROOT, "paper_1806_01422_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def algorithmic_flops_per_element(op, d, n):
    """Sum-factorised FLOPs of one element (naive n-term contractions, 2 flop per multiply-add).

    F : 2d^2 contractions (d gradients and d divergences per component) + advection (2d flop per
        node and component) + the subtraction (1);  J, J^T: 3d^2 contractions + 4d^2 + d per node.
    """
    contr = 2 * n ** (d + 1)
    if op == "rhs":
        return 2 * d * d * contr + (2 * d * d + d) * n ** d
    return 3 * d * d * contr + (4 * d * d + d) * n ** d


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[2:]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- oracle leg
# The oracle's operators with the element loop split over the host cores (the cpu_baseline and
# --impl reference legs only).  The oracle itself is unchanged: each worker of a fork pool, started
# inside a CUDA-free child process, applies the oracle's element-local operator (Grid.local_rhs,
# Grid.local_jacT) to a contiguous range of element slabs along the slowest array axis and sums
# the element-local values into its own slab of the global array.  It writes the slab's interior
# planes to the shared output and hands its two end planes to the parent, which adds the planes
# that neighbouring slabs share, in a fixed order.  The definitions are those of Grid.rhs and
# Grid.jacT; only the grouping of the gather-scatter sum differs.
_POOL = {}


def _shared_array(n):
    import mmap
    import numpy as np
    return np.frombuffer(mmap.mmap(-1, max(8, 8 * n)), dtype=np.float64, count=n)


def _slab_index(g, a, b):
    """Element ids of slabs [a, b) and their index tuple into a local array of (b-a) N + 1 planes."""
    import numpy as np
    d, E, N, n = g.d, g.E, g.N, g.n
    per_slab = E ** (d - 1)
    elems = np.arange(a * per_slab, b * per_slab)
    ec = np.unravel_index(elems, (E,) * d)          # array order, slowest axis first
    idx = []
    for p in range(d):
        shape = [1] * (1 + d)
        shape[0] = len(elems)
        shape[1 + p] = n
        if p == 0:
            v = (ec[0][:, None] - a) * N + np.arange(n)[None, :]
        else:
            v = (ec[p][:, None] * N + np.arange(n)[None, :]) % g.G
        idx.append(v.reshape(shape))
    return elems, tuple(idx)


def _pool_task(task):
    import numpy as np
    op, k = task
    P = _POOL
    g = P["grid"]
    a, b = P["slabs"][k]
    elems, idx = P["index"][k]
    d, N, G = g.d, g.N, g.G
    shp = (d,) + g.global_shape()
    u = P["in0"].reshape(shp)
    if op == "rhs":
        R = g.local_rhs(g.gather_vec(u, elems))
    else:
        v = P["in1"].reshape(shp)
        Mloc = g.gather(g.M, elems)
        Z = np.stack([g.gather(v[c], elems) / Mloc for c in range(d)])   # Q M^-1 v, node by node
        R = g.local_jacT(g.gather_vec(u, elems), Z)
    loc = np.zeros((d, (b - a) * N + 1) + (G,) * (d - 1))
    for c in range(d):
        np.add.at(loc[c], idx, R[c])
    out = P["out"].reshape(shp)
    lo, hi = a * N, b * N
    out[:, lo + 1:hi] = loc[:, 1:-1] / g.M[lo + 1:hi] if op == "rhs" else loc[:, 1:-1]
    bnd = P["bnd"].reshape((len(P["slabs"]), 2, d) + (G,) * (d - 1))
    bnd[k, 0] = loc[:, 0]
    bnd[k, 1] = loc[:, -1]
    return k


class OraclePool:
    """Grid.rhs and Grid.jacT of the oracle, with the element loop split over `procs` processes.

    Create it in a process that has not initialised CUDA (a fork after CUDA init can hang);
    bench.py does so in a child process with no visible GPU.
    """

    def __init__(self, g, procs):
        import multiprocessing as mp
        procs = max(1, min(int(procs), g.E))
        bounds = [round(i * g.E / procs) for i in range(procs + 1)]
        slabs = [(bounds[i], bounds[i + 1]) for i in range(procs)]
        n = g.ndof()
        plane = g.d * g.G ** (g.d - 1)
        _POOL.clear()
        _POOL.update(grid=g, slabs=slabs, index=[_slab_index(g, a, b) for a, b in slabs],
                     in0=_shared_array(n), in1=_shared_array(n), out=_shared_array(n),
                     bnd=_shared_array(procs * 2 * plane))
        self.g, self.procs, self.slabs = g, procs, slabs
        self.pool = mp.get_context("fork").Pool(procs)

    def close(self):
        self.pool.terminate()
        self.pool.join()

    def _run(self, op):
        import numpy as np
        g, N = self.g, self.g.N
        self.pool.map(_pool_task, [(op, k) for k in range(self.procs)])
        shp = (g.d,) + g.global_shape()
        out = _POOL["out"].reshape(shp)
        bnd = _POOL["bnd"].reshape((self.procs, 2, g.d) + (g.G,) * (g.d - 1))
        for k, (a, _) in enumerate(self.slabs):
            s = bnd[k, 0] + bnd[(k - 1) % self.procs, 1]
            out[:, a * N] = s / g.M[a * N] if op == "rhs" else s
        return np.array(out)

    def rhs(self, u):
        _POOL["in0"][:] = u.ravel()
        return self._run("rhs")

    def jacT(self, u, v):
        _POOL["in0"][:] = u.ravel()
        _POOL["in1"][:] = v.ravel()
        return self._run("jacT")

    def objective(self, u, u_obs):
        return self.g.objective(u, u_obs)


def oracle_sample(workload, rk_steps, reps, procs):
    """Seconds of `reps` oracle gradient evaluations of `rk_steps` steps each (child process)."""
    import numpy as np
    from oracle.sem import Grid
    from oracle import rk as ork
    from paper_1806_01422_gb300 import inputs
    w = WORKLOADS[workload]
    g = Grid(w["dim"], w["E"], w["N"], w["nu"])
    x = g.coords()
    u0, uo = inputs.workload_field(w["dim"], x, inputs.SEED_U0), inputs.workload_field(w["dim"], x, inputs.SEED_UOBS)
    pg = OraclePool(g, procs)
    secs, J, finite = [], None, True
    try:
        for _ in range(reps):
            t0 = time.perf_counter()
            J, lam, _ = ork.objective_and_gradient(pg, u0, uo, w["dt"], rk_steps, w["scheme"])
            secs.append(time.perf_counter() - t0)
            finite = finite and bool(np.isfinite(lam).all())
    finally:
        pg.close()
    return {"seconds": secs, "rk_steps": rk_steps, "procs": pg.procs, "J": J, "finite": finite}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_oracle_child(workload, rk_steps, reps=1, procs=None):
    env = dict(os.environ)
    # one BLAS thread per worker process: the pool supplies the parallelism
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    procs = procs or host_cores()
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-sample", workload, str(rk_steps), str(reps),
           str(procs)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: %s" % r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(workload, target_s=15.0):
    """Oracle gradient evaluations/s from a bounded sample on all host cores, scaled to the full horizon."""
    w = WORKLOADS[workload]
    cores = host_cores()
    if w["scheme"] == "cn":
        return {"value": None, "unit": "gradient evals/s", "cores": cores, "kind": "oracle",
                "sample": "none: the oracle's Crank-Nicolson solves assemble dense Jacobians, which do not fit "
                          "at %s" % w["desc"].split(", ")[2]}
    probe = run_oracle_child(workload, 1, 1, cores)
    per_step = max(probe["seconds"][0], 1e-6)
    n = int(max(1, min(w["nsteps"], target_s / per_step)))
    res = run_oracle_child(workload, n, 1, cores)
    per_eval = res["seconds"][0] * w["nsteps"] / n
    return {"value": 1.0 / per_eval, "unit": "gradient evals/s", "cores": res["procs"], "kind": "oracle",
            "sample": "%d of %d RK steps of one gradient evaluation (forward + misfit + adjoint over the stored "
                      "stages), FP64 numpy oracle with its element loop split over %d processes; time scaled by "
                      "%d/%d" % (n, w["nsteps"], res["procs"], w["nsteps"], n),
            "seconds": res["seconds"][0]}


# ---------------------------------------------------------------- distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=os.environ.get("BENCH_BACKEND", "nccl"))
    return world, rank, local


def max_over_ranks(value, world, device):
    """Max of a float over all ranks (the slowest rank sets the job time)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(per_rank_seconds, steps, world, device):
    """Whole-job throughput: all ranks' steps over the slowest rank's time (weak scaling)."""
    tmax = max_over_ranks(per_rank_seconds, world, device)
    return world * steps / tmax, tmax


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- arms
def reference_arm(args, world, rank):
    """The oracle (the slow plain CPU program the path is checked against), as it stands."""
    if rank != 0:
        return None
    w = WORKLOADS[args.workload]
    if w["scheme"] == "cn":
        return {"impl": "reference", "unavailable": "the oracle's Crank-Nicolson solves assemble dense Jacobians, "
                                                    "which do not fit at 401,408 unknowns"}
    n = args.oracle_rk_steps or w.get("oracle_steps", 10)
    res = run_oracle_child(args.workload, n, args.warmup + args.steps)
    secs = res["seconds"][args.warmup:]
    per_eval = statistics.mean(secs) * w["nsteps"] / n
    value = 1.0 / per_eval
    cores = res["procs"]
    sample = ("each step: %d of %d RK steps of one gradient evaluation (forward + misfit + adjoint over the "
              "stored stages), FP64 numpy oracle with its element loop split over %d processes; time scaled "
              "by %d/%d" % (n, w["nsteps"], cores, w["nsteps"], n))
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "gradient evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_eval * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": w["data"], "config": {"workload": w["desc"]},
            "cpu_baseline": {"value": value, "unit": "gradient evals/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "gradient evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def roofline_of(prof, args, w, s, precision):
    """Roofline of the dominant kernel kind from the sampled CUDA-event times of a timed region."""
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms, dom_n, dom_bytes = kinds[dom]
    avg_s = dom_ms / dom_n / 1e3
    fp32 = precision == "fp32_bulk"
    names = {"rhs": "rhs", "jac": "jac", "jacT": "jact"}
    if args.workload == "batch":
        shapes = list(zip(s.E, s.N))
        kname = "batch_elem2_kernel"
    else:
        shapes = [(w["E"], w["N"])]
        kname = None
    if dom == "assemble":
        # gather-scatter: the d E^d (N+1)^d element-local values read once, and per unknown each
        # RK-epilogue source read and each output written once (8 B each); the library sums these
        # bytes over the timed launches, whose epilogues differ from stage to stage
        achieved = dom_bytes / (dom_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": args.hbm_peak, "unit": "GB/s",
                "frac": achieved / args.hbm_peak, "kernel": "assemble kernel"}
    else:
        flops = sum(algorithmic_flops_per_element(dom, w["dim"], N + 1) * E ** w["dim"] for E, N in shapes)
        achieved = flops / avg_s / 1e12
        dfk = precision == "fp64_df"
        peak = PEAK_FP32_TFLOPS if fp32 else (PEAK_DF_TFLOPS if dfk else PEAK_FP64_TFLOPS)
        ctype = "float" if fp32 else ("semk::dfa::dfloat" if dfk else "double")
        kernel = kname or "%s%d_kernel<%s,%d>" % (names[dom], w["dim"], ctype, w["N"] + 1)
        if w["dim"] == 3 and ctype == "double" and w["N"] == 7 and not kname:
            kernel = "%s3_f64_kernel<8>" % names[dom]     # the register-capped FP64 n = 8 kernels
        if dfk and w["dim"] == 2:
            kernel = "op2c_kernel<%s,%d> (%s)" % (ctype, w["N"] + 1, {"rhs": "F", "jac": "J", "jacT": "J^T"}[dom])
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "kernel": kernel}
        if dfk:
            roof["peak_note"] = ("double-float multiply-add rate of the FP32 pipe: 152 SMs x 128 lanes x 2.07 GHz "
                                 "/ 13 FP32 operations per multiply-add, x 2 flop")
        # the second roof: the operator's minimum HBM bytes per launch (16 B per unknown for F: u in, F out;
        # 24 B for J and J^T: two inputs, one output) over the same launch time
        ndof = sum(w["dim"] * (E * N) ** w["dim"] for E, N in shapes)
        alg_bytes = (16 if dom == "rhs" else 24) * ndof
        hbm = alg_bytes / avg_s / 1e9
        roof["hbm"] = {"algorithmic_bytes": alg_bytes, "achieved": hbm, "peak": args.hbm_peak, "unit": "GB/s",
                       "frac": hbm / args.hbm_peak}
    key = "%s@%s@%s" % (roof["kernel"], args.workload, precision)
    tr = TRAFFIC.get(key)
    tr_ok = tr and tr["src"] == kernel_src_hash("assemble" if dom == "assemble" else "elem")
    roof["traffic"] = tr["bytes"] if tr_ok else None
    if tr_ok:
        roof["traffic_source"] = tr["capture"]
    if roof["bound"] == "alu":
        roof["note"] = ("achieved counts the algorithmic flops of plain n-term contractions; the kernels split "
                        "each contraction into even and odd halves (n^2/2 + n operations per line), so frac can "
                        "exceed the fraction of FP pipe cycles ncu reports")
    roof["avg_launch_us"] = avg_s * 1e6
    roof["timed_launches"] = dom_n
    roof["timing"] = "CUDA events around 1 in %d launches of each kernel kind, on the launching stream%s, " \
                     "inside the timed region" % (args.profile_every,
                                                  "" if args.no_graph else " (event nodes of the replayed graph)")

    return roof


def measure_form(args, w, precision, u0, uo, grad_ref, J_ref, dev):
    """Gradient evaluations/s of another precision form on the same inputs (same timing rules), its
    dominant kernel's roofline, and its misfit and gradient against the FP64 form's."""
    import torch
    from paper_1806_01422_gb300 import Sem
    s = Sem(w["dim"], w["E"], w["N"], w["nu"], precision=precision, ckpt=w["ckpt"], ckpt_slots=w["slots"],
            device=dev)
    g = s.empty()
    s.use_graph(not args.no_graph)
    s.profile(args.profile_every)
    reps = max(1, min(args.steps, args.extra_reps))
    for _ in range(2):
        J, _ = s.objective_grad(u0, uo, w["dt"], w["nsteps"], w["scheme"], grad=g)
    s.profile_read(reset=True)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        J, _ = s.objective_grad(u0, uo, w["dt"], w["nsteps"], w["scheme"], grad=g)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    s.profile(0)
    prof = s.profile_read(reset=True)
    elapsed = e0.elapsed_time(e1) / 1e3
    roof = roofline_of(prof, args, w, s, precision)
    out = {"value": reps / elapsed, "ms_per_step": elapsed / reps * 1e3, "reps": reps,
           "J_rel_diff_vs_fp64": abs(J - J_ref) / abs(J_ref),
           "grad_rel_err_vs_fp64": float((g - grad_ref).abs().max() / grad_ref.abs().max()),
           "roofline": {k: roof[k] for k in ("bound", "achieved", "peak", "unit", "frac", "kernel", "avg_launch_us")}}
    s.close()
    return out


def gpu_arm(args, world, rank, local):
    import torch
    from paper_1806_01422_gb300 import Sem, inputs
    from paper_1806_01422_gb300 import _lib as L

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = WORKLOADS[args.workload]
    if args.workload == "batch":
        from paper_1806_01422_gb300 import SemBatch
        Es, Ns = inputs.batch_shapes(w["count"])
        s = SemBatch(Es, Ns, [w["nu"]] * w["count"], ckpt=w["ckpt"], device=dev)
        u0_h = torch.from_numpy(s.pack([inputs.field_2d(s.coords(k), inputs.batch_seeds(k)[0])
                                        for k in range(s.count)])).pin_memory()
        uo_h = torch.from_numpy(s.pack([inputs.field_2d(s.coords(k), inputs.batch_seeds(k)[1])
                                        for k in range(s.count)])).pin_memory()
        units = w["count"]
    else:
        s = Sem(w["dim"], w["E"], w["N"], w["nu"], precision=args.precision, ckpt=w["ckpt"], ckpt_slots=w["slots"],
                device=dev)
        if args.contraction != "cuda_core":
            s.set_contraction(args.contraction)
        x = s.coords()
        u0_h = torch.from_numpy(inputs.workload_field(w["dim"], x, inputs.SEED_U0)).pin_memory()
        uo_h = torch.from_numpy(inputs.workload_field(w["dim"], x, inputs.SEED_UOBS)).pin_memory()
        units = 1
    u0, uo = u0_h.to(dev), uo_h.to(dev)
    grad = s.empty()
    nsteps, dt, scheme = w["nsteps"], w["dt"], w["scheme"]
    if scheme == "cn":
        args.no_graph = True    # the implicit solves synchronise with the host: never captured

    def step():
        return s.objective_grad(u0, uo, dt, nsteps, scheme, grad=grad)

    # the gradient evaluation runs as one CUDA graph (recorded by the first warm-up call,
    # with the sampled kernel-timing events inside it)
    if not args.no_graph:
        s.use_graph(True)
    s.profile(args.profile_every)
    graph_note = None
    try:
        for _ in range(args.warmup):
            J, _ = step()
        s.profile_read(reset=True)
    except L.SemError as e:
        if args.no_graph:
            raise
        # timed event nodes inside the graph were refused: measure stream launches instead
        graph_note = "graph replay with timed event nodes failed (%s); stream launches measured" % e
        s.use_graph(False)
        args.no_graph = True
        s.profile(args.profile_every)
        for _ in range(args.warmup):
            J, _ = step()
        s.profile_read(reset=True)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier(world)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            J, _ = step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
    s.profile(0)
    prof = s.profile_read(reset=True)
    st = s.sweep_stats()
    elapsed = e0.elapsed_time(e1) / 1e3
    value, tmax = job_value(elapsed, args.steps * units, world, dev)
    # element kernels and assemblies (counted by the library; fused assemblies are not
    # launches), plus misfit, partial sum and adjoint seed per step
    if args.workload == "batch":
        launches = args.steps * (2 * (st["forward_rhs"] + st["adjoint_rhs"] + st["adjoint_jacT"]) + 3)
    else:
        launches = args.steps * (s.launch_count() + 3)
    if scheme == "cn":
        # per Arnoldi step 5 two-kernel dot passes, 2 axpys and a scale; per GMRES solve a norm, a
        # scale and the update; per Newton iteration the update and two norms
        cs = s.solver_stats()
        krylov = cs["forward_krylov"] + cs["adjoint_krylov"]
        launches = args.steps * (2 * cs["applies"] + 13 * krylov + 4 * (cs["newton"] + nsteps)
                                 + 5 * cs["newton"] + 3)

    roof = roofline_of(prof, args, w, s, args.precision)
    fp32 = args.precision == "fp32_bulk"

    unit = "instance gradient evals/s" if args.workload == "batch" else "gradient evals/s"
    stages = {"rk4": 4, "ssprk3": 3, "euler": 1, "cn": 1}[scheme]
    traj_gb = s.ndof * 8 / 1e9 * {"stages": nsteps * stages, "states": nsteps + (scheme == "cn"),
                                  "binomial": w["slots"]}.get(w["ckpt"], nsteps)
    out = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": tmax / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else ("f32x2 (double-float element kernels; f64 states and reductions)"
                                                if args.precision == "fp64_df" else "f64"), "data": w["data"],
           "config": {"workload": w["desc"], "dim": w["dim"], "E": w["E"], "N": w["N"], "unknowns": s.ndof,
                      "instances": units,
                      "scheme": scheme, "dt": dt, "rk_steps": nsteps, "trajectory": w["ckpt"],
                      "precision": args.precision, "contraction": args.contraction,
                      "parallelism": "replicas" if world > 1 else "single GPU",
                      "l2": "inputs larger than L2: every step writes and re-reads the stored trajectory "
                            "(%.1f GB: %s)" % (traj_gb, w["ckpt"])},
           "roofline": roof, "gpu_launches": launches, "clocks": clk.summary(), "J": J,
           **({"horizon": w["horizon"]} if "horizon" in w else {}),
           "execution": graph_note or ("stream launches" if args.no_graph else "CUDA graph replay (sem_set_graph)"),
           "kernel_ms_per_step": {k: v[0] * args.profile_every / args.steps for k, v in prof.items()}}
    if scheme == "cn":
        out["solver"] = dict(s.solver_stats(), note="counters of the last gradient evaluation")

    if rank == 0 and not args.no_extras and args.precision == "fp64" and w["scheme"] != "cn" \
            and args.workload != "batch":
        # the other precision forms on the same inputs, reported against this FP64 form
        out["forms"] = {p: measure_form(args, w, p, u0, uo, grad, J, dev) for p in ("fp64_df", "fp32_bulk")}
    if rank == 0 and not args.no_extras:
        out.update(extras(s, u0, uo, w, dev))
        # end to end through the public API with host buffers (pinned), copies inside the timed region
        reps = max(1, min(args.steps, args.extra_reps))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(reps):
            Jh, gh = s.objective_grad(u0_h, uo_h, dt, nsteps, scheme, host=True)
        t1 = time.perf_counter()
        out["e2e"] = {"value": reps * units / (t1 - t0), "unit": unit, "reps": reps,
                      "h2d_bytes_per_step": 2 * s.ndof * 8, "d2h_bytes_per_step": s.ndof * 8 + 8}
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_seconds)
    if rank == 0 and args.lbfgs and args.workload != "batch":
        out["lbfgs"] = lbfgs_run(s, w, args.lbfgs, dev)
    return out if rank == 0 else None


def lbfgs_run(s, w, iters, dev):
    """The optimisation loop of Fig. 1: recover the initial condition that produced u_obs.

    u_obs is the final state of the forward sweep from the seed-2 field; the search starts
    from the seed-1 field.  Outside the timed region.
    """
    import torch
    from paper_1806_01422_gb300 import inputs
    from paper_1806_01422_gb300.inverse import recover_initial_condition
    x = s.coords()
    u_true = torch.from_numpy(inputs.workload_field(w["dim"], x, inputs.SEED_UOBS)).to(dev)
    u_init = torch.from_numpy(inputs.workload_field(w["dim"], x, inputs.SEED_U0)).to(dev)
    s.use_graph(False)   # every evaluation point is a new tensor: stream launches, no re-recording
    u_obs = s.rk_forward(u_true, w["dt"], w["nsteps"], w["scheme"]).clone()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    est, hist = recover_initial_condition(s, u_obs, u_init, w["dt"], w["nsteps"], w["scheme"], iters=iters)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    rel = lambda a: float((a - u_true).norm() / u_true.norm())
    return {"iterations": hist[-1][0], "gradient_evals": hist[-1][3], "seconds": t1 - t0,
            "J_first": hist[0][1], "J_last": hist[-1][1], "grad_norm_first": hist[0][2], "grad_norm_last": hist[-1][2],
            "u0_rel_error_first": rel(u_init), "u0_rel_error_last": rel(est),
            "J_history": [h[1] for h in hist]}


def median_ms(fn, reps=30, warm=5, min_batch_ms=1.0):
    """Median over reps repetitions of the CUDA-event time (ms) of one call of fn, after warm calls.
    Each repetition times a batch of calls long enough (min_batch_ms) that the events' resolution
    (about 0.5 us) does not matter, and divides by the batch size; the events are recorded on the
    current stream between consecutive batches."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    inner = max(1, int(math.ceil(min_batch_ms / max(e0.elapsed_time(e1) / 3, 1e-3))))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for i in range(reps):
        for _ in range(inner):
            fn()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    return statistics.median(ev[i].elapsed_time(ev[i + 1]) / inner for i in range(reps))


def extras(s, u0, uo, w, dev):
    """Standalone operator throughput and the forward/adjoint split (outside the timed region)."""
    import torch
    stream = torch.cuda.current_stream(dev)
    out = s.empty()

    tf = median_ms(lambda: s.rhs(u0, out))
    tt = median_ms(lambda: s.jacT(u0, uo, out))
    uN = s.empty()
    lam = s.empty()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize(dev)
    e[0].record(stream)
    s.rk_forward(u0, w["dt"], w["nsteps"], w["scheme"], out=uN)
    e[1].record(stream)
    s.objective(uN, uo, lam)
    s.rk_adjoint(lam, out=lam)
    e[2].record(stream)
    torch.cuda.synchronize(dev)
    fwd, adj = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    return {"gdofs_F": s.ndof / tf / 1e6, "gdofs_JT": s.ndof / tt / 1e6, "JT_over_F_apply": tt / tf,
            "forward_ms": fwd, "adjoint_ms": adj, "adjoint_forward_ratio": adj / fwd}


def order_sweep(precisions=("fp64", "fp64_df", "fp32_bulk"), target=34e6, reps=20):
    """Standalone F(u) and J^T v throughput over orders N at about `target` 3D unknowns (median of
    reps applies)."""
    import torch
    from paper_1806_01422_gb300 import Sem, inputs
    rows = []
    for prec in precisions:
        for N in (3, 5, 7, 9, 11, 13, 15):
            E = max(2, int(round((target / 3) ** (1 / 3) / N)))
            s = Sem(3, E, N, 5e-4, precision=prec)
            x = s.coords()
            u = torch.from_numpy(inputs.field_3d(x, inputs.SEED_U0)).cuda()
            v = torch.from_numpy(inputs.field_3d(x, inputs.SEED_UOBS)).cuda()
            out = s.empty()
            res = {}
            for name, fn in (("F", lambda: s.rhs(u, out)), ("JT", lambda: s.jacT(u, v, out))):
                ms = median_ms(fn, reps=reps, warm=3)
                res[name] = {"ms": ms, "gdofs": s.ndof / ms / 1e6}
            rows.append({"precision": prec, "N": N, "E": E, "unknowns": s.ndof, **res,
                         "JT_over_F": res["JT"]["ms"] / res["F"]["ms"]})
            print(json.dumps(rows[-1]), flush=True)
            del s, u, v, out
            torch.cuda.empty_cache()
    return rows


def contraction_ab(reps=20):
    """Standalone F(u) at 16^3 hexes, N = 15 with each contraction engine and precision: apply time,
    sampled element-pass and assembly times, and the result against the CUDA-core engine."""
    import torch
    from paper_1806_01422_gb300 import Sem, inputs
    rows = []
    for prec in ("fp64", "fp32_bulk"):
        s = Sem(3, 16, 15, 2e-4, precision=prec)
        u = torch.from_numpy(inputs.field_3d(s.coords(), inputs.SEED_U0)).cuda()
        out = s.empty()
        ref = None
        for mode in ("cuda_core", "tensor"):
            s.set_contraction(mode)
            ms = median_ms(lambda: s.rhs(u, out), reps=reps, warm=3)
            s.profile(1)
            for _ in range(reps):
                s.rhs(u, out)
            torch.cuda.synchronize()
            s.profile(0)
            prof = s.profile_read(reset=True)
            if ref is None:
                ref = out.clone()
            row = {"precision": prec, "contraction": mode, "F_ms": ms, "gdofs_F": s.ndof / ms / 1e6,
                   "elem_us": prof["rhs"][0] / max(prof["rhs"][1], 1) * 1e3,
                   "assemble_us": prof["assemble"][0] / max(prof["assemble"][1], 1) * 1e3,
                   "rel_diff_vs_cuda_core": float((out - ref).abs().max() / ref.abs().max())}
            rows.append(row)
            print(json.dumps(row), flush=True)
        s.close()
        del u, out
        torch.cuda.empty_cache()
    return rows


def ops_once(dim, E, N, precision, contraction="cuda_core"):
    """One F and one J^T apply (for ncu captures of the element and assembly kernels)."""
    import torch
    from paper_1806_01422_gb300 import Sem, inputs
    s = Sem(dim, E, N, 1e-3, precision=precision)
    if contraction != "cuda_core":
        s.set_contraction(contraction)
    x = s.coords()
    u = torch.from_numpy(inputs.workload_field(dim, x, inputs.SEED_U0)).cuda()
    v = torch.from_numpy(inputs.workload_field(dim, x, inputs.SEED_UOBS)).cuda()
    out = s.empty()
    s.rhs(u, out)
    s.jacT(u, v, out)
    torch.cuda.synchronize()
    print(json.dumps({"ops_once": [dim, E, N, precision, contraction], "unknowns": s.ndof}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="3d", choices=sorted(WORKLOADS))
    ap.add_argument("--extra-reps", type=int, default=3,
                    help="timed repetitions of the other precision forms and of the end-to-end leg (at most --steps)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_bulk", "fp64_df"])
    ap.add_argument("--contraction", default="cuda_core", choices=["cuda_core", "tensor"],
                    help="element-kernel contraction engine (tensor: 3D, N=15 only)")
    ap.add_argument("--contraction-ab", action="store_true",
                    help="A/B of the contraction engines: standalone F at 16^3 hexes, N=15, FP64 and FP32-bulk")
    ap.add_argument("--hbm-peak", type=float, default=None, help="GB/s; default: MEASURED_PEAKS.json")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--oracle-rk-steps", type=int, default=None,
                    help="RK steps per oracle sample of the reference arm (default: the workload's own)")
    ap.add_argument("--rk-steps", type=int, default=None,
                    help="override the workload's RK step count (profiling runs only; not a bench number)")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--lbfgs", type=int, default=0, metavar="K",
                    help="after the timed region, run K L-BFGS iterations recovering u0 (single-instance workloads)")
    ap.add_argument("--profile-every", type=int, default=64, help="time one launch in this many per kernel kind")
    ap.add_argument("--no-graph", action="store_true", help="launch on the stream instead of replaying a CUDA graph")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-sample", nargs=4, metavar=("WORKLOAD", "RK_STEPS", "REPS", "PROCS"),
                    help=argparse.SUPPRESS)
    ap.add_argument("--order-sweep", action="store_true",
                    help="standalone 3D F and J^T throughput over N in {3,5,7,9,11,15} at ~34M unknowns")
    ap.add_argument("--ops-once", nargs=4, metavar=("DIM", "E", "N", "PRECISION"),
                    help="for ncu: one F and one J^T apply on the workload field of that size, no timing")
    args = ap.parse_args()

    if args.oracle_sample:
        wl, k, reps, procs = args.oracle_sample
        print(json.dumps(oracle_sample(wl, int(k), int(reps), int(procs))))
        return
    if args.order_sweep:
        order_sweep()
        return
    if args.contraction_ab:
        contraction_ab()
        return
    if args.ops_once:
        ops_once(int(args.ops_once[0]), int(args.ops_once[1]), int(args.ops_once[2]), args.ops_once[3],
                 args.contraction)
        return
    if args.rk_steps:
        for w in WORKLOADS.values():
            w["nsteps"] = args.rk_steps
    if args.hbm_peak is None:
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
                args.hbm_peak = float(json.load(fh)["hbm_gbs"])
        except (OSError, KeyError, ValueError):
            args.hbm_peak = 6800.0
    world, rank, local = dist_setup()
    if args.impl == "reference":
        res = reference_arm(args, world, rank)
    else:
        res = gpu_arm(args, world, rank, local)
    if res is not None:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
