#!/usr/bin/env python3
"""Benchmark of the GB300 HPS solver on the variable-coefficient workload: 64 x 64 leaves,
p = 16 (q = 15), seeded 8-mode Fourier-series coefficients, a batch of nrhs right-hand
sides.

One step is one pass of the whole hot path over one batch:
  FP64 build (leaf eliminations + merges), FP64 solve of the batch, the adjoint of the
  batch (gradients of J = 0.5 ||u - u_obs||^2 w.r.t. f, g and the six coefficient
  fields), then the mixed-precision build and the mixed solve (FP32 sweeps refined
  against double-float residuals to an estimated error below 1e-9 max|u|).
value = solved degrees of freedom (leaf-major n_leaf p^2 per right-hand side) per second
of step time, whole job.  Phase timings give build seconds, solve DOF/s (FP64 vs mixed)
and the gradient/forward ratio.

Beside the headline line (extra keys, outside the timed region): solve-only throughput and
the solve roofline at nrhs 1, 8 and 64; the other workloads (Poisson 4 x 4, the locally
refined L-shape, backward-Euler heat stepping on 128 x 128 leaves, the adjoint with leaf
recomputation, orders p = 16 .. 30); and the CPU oracle timed on the full workload.

--impl reference times the CPU oracle (FP64 NumPy restatement of the method) on a bounded
sample of the workload instead.  Launch with torchrun for several GPUs: every rank solves
its own replica (no data-path collective).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

# the CPU oracle's BLAS uses every host core; set before NumPy loads its BLAS
_NCPU = str(os.cpu_count() or 1)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, _NCPU)

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = 64
P = 16
METRIC = "build s & solve DOF/s at 1e-8 rel err: mixed vs FP64 GPU; grad/forward ratio"
UNIT = "DOF/s"
# FP64 FFMA peak of GB300: 152 SMs x 2 FP64 FMA/clock/SM x 2 flop x 2070 MHz (the 1.25
# TFLOP/s FP64 figure at the maximum SM clock); no FP64 tensor path is faster on this part.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# FP32 FFMA peak: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--nrhs", type=int, default=64)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads (configs 1, 3, 4, 5, p-sweep)")
    ap.add_argument("--heat-steps", type=int, default=100,
                    help="backward-Euler steps of the heat workload (1000 in full; fewer are extrapolated)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="fixed tile rules instead of the autotuner (profiling captures of a chosen launch)")
    ap.add_argument("--nx", type=int, default=64, help="leaves per side (64 is the benchmark workload; "
                    "smaller values are for profiling captures)")
    args = ap.parse_args()
    global NX
    NX = args.nx
    return args


def workload():
    return "varcoef-%dx%d-p%d" % (NX, NX, P)


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------
# workload (inputs from the seeded synthetic generators at the library's node coordinates)

def make_inputs(tree, nrhs, p=P):
    import synthetic as syn
    cheb = tree.nodes(p, p - 1, "cheb")
    bnd = tree.nodes(p, p - 1, "boundary")
    nl = cheb.shape[0] // (p * p)
    X = cheb[:, 0].reshape(nl, p * p)
    Y = cheb[:, 1].reshape(nl, p * p)
    prob = syn.VarCoeffProblem()
    coeffs = np.ascontiguousarray(np.array(prob.coeffs(X, Y)))
    c_obs = np.ascontiguousarray(np.array(prob.coeffs(X, Y, perturbed=True)))
    g0 = prob.load(X, Y)
    f0 = prob.dirichlet(bnd[:, 0], bnd[:, 1])
    scale = np.linspace(0.5, 1.5, nrhs)
    g = np.ascontiguousarray(g0[..., None] * scale)
    f = np.ascontiguousarray(f0[:, None] * scale)
    return coeffs, c_obs, f, g


# ------------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def traffic_record(kernel):
    """DRAM bytes per launch of a kernel from the committed ncu summary, if the kernel
    source has not changed since the capture (source hash recorded with it)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel:
            src = os.path.join(ROOT, "paper_1612_02736_gb300", "csrc", parts[2])
            if not os.path.exists(src):
                return None
            h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
            return float(parts[1]) if h == parts[3] else None
    return None


def timed(stream, fn, reps=1):
    """Milliseconds per call of fn() between CUDA events on stream (synchronised)."""
    import torch
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        out = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps, out


# ------------------------------------------------------------------------------------
# solve roofline: algorithmic bytes of one solve (every stored operator entry read once per
# sweep; the residual passes of the mixed path read the six coefficient fields, u and g and
# write r) and the FLOPs of its products, against the measured HBM copy bandwidth and the
# FP64 / FP32 FFMA peaks

def solve_roofline(s, nrhs, ms, iters, hbm_gbs):
    n_nodes = s.n_leaf * s.p * s.p
    vec = 2.0 * n_nodes * nrhs * 8 + s.n_bdry * nrhs * 8       # g in, u out, f in
    if s.precision == "fp64":
        sweeps, esize, res = 1, 8, 0.0
    else:
        sweeps, esize = 1 + iters, 4
        res = iters * (6.0 * n_nodes * 8 + 3.0 * n_nodes * nrhs * 8)
    entries = s.operator_bytes / esize
    byts = sweeps * s.operator_bytes + res + vec
    flops = 2.0 * entries * nrhs * sweeps
    sec = ms / 1e3
    gbs = byts / sec / 1e9
    out = {"ms": ms, "dof_per_s": n_nodes * nrhs / sec, "sweeps": sweeps, "bytes": byts, "achieved_gbs": gbs,
           "hbm_frac": gbs / hbm_gbs, "tflops": flops / sec / 1e12}
    if s.precision == "fp64":
        out["fp64_pipe_frac"] = out["tflops"] / FP64_PEAK_TFLOPS
        out["bound"] = ("fp64 pipe (2 FP64 FMA/clk/SM: at one FMA per 8-byte entry and rhs it caps the "
                        "sweep at %.2f of HBM at nrhs 1)" % (152 * 2 * 2.070e9 * 8 / 1e9 / hbm_gbs / nrhs)
                        if nrhs <= 4 else "tensor-core FP64 digit products (9 digit planes per entry)")
    else:
        out["fp32_pipe_frac"] = out["tflops"] / FP32_PEAK_TFLOPS
        out["bound"] = ("hbm" if nrhs <= 8 else
                        "bf16 tensor-core piece products (3 pieces per FP32 entry) and the double-float residual")
    return out


# ------------------------------------------------------------------------------------

def run_gpu(args, rank, world, local):
    import torch
    from paper_1612_02736_gb300 import Solver, Tree, build, _native

    torch.cuda.set_device(local)
    build.build()
    lib = _native.load()
    tree = Tree.uniform(0.0, 0.0, 1.0, 1.0, NX, NX)
    nrhs = args.nrhs
    coeffs_h, cobs_h, f_h, g_h = make_inputs(tree, nrhs)
    dev = torch.device("cuda", local)
    coeffs = torch.from_numpy(coeffs_h).to(dev)
    f = torch.from_numpy(f_h).to(dev)
    g = torch.from_numpy(g_h).to(dev)
    n_leaf = NX * NX
    dof = n_leaf * P * P * nrhs
    # observation for the misfit: FP64 solution with the perturbed coefficients
    s_obs = Solver(tree, torch.from_numpy(cobs_h).to(dev), P, "fp64")
    u_obs = s_obs.solve(f, g)
    s_obs.close()
    del s_obs

    stream = torch.cuda.current_stream()
    # tile autotuner: the warm-up steps tune every launch shape once (kept in memory)
    tune = not args.no_autotune

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        return e

    def step(coeffs, f, g, record):
        t = [ev()]
        s64 = Solver(tree, coeffs, P, "fp64", autotune=tune)
        t.append(ev())
        u64 = s64.solve(f, g)
        t.append(ev())
        fb, gb, cb = s64.adjoint(u64 - u_obs, u=u64)
        t.append(ev())
        sm = Solver(tree, coeffs, P, "mixed", autotune=tune)
        t.append(ev())
        um = sm.solve(f, g)
        t.append(ev())
        iters = sm.last_iters
        s64.close()
        sm.close()
        if record is not None:
            record.append((t, iters))
        return u64, um, fb, gb, cb

    for _ in range(args.warmup):
        step(coeffs, f, g, None)
    torch.cuda.synchronize()
    u64, um, *_ = step(coeffs, f, g, None)
    torch.cuda.synchronize()
    rel_err = float((um - u64).abs().max() / u64.abs().max())

    # ---- device-resident timed region
    recs = []
    lib.hps_timing_reset()
    lib.hps_timing_enable(1)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0 = ev()
        for _ in range(args.steps):
            step(coeffs, f, g, recs)
        e1 = ev()
        torch.cuda.synchronize()
    barrier(world)
    lib.hps_timing_enable(0)
    total_ms = allmax(e0.elapsed_time(e1), world)
    table = _native.timing_table()
    phases = np.zeros(5)
    iters = []
    for t, it in recs:
        phases += np.array([t[i].elapsed_time(t[i + 1]) for i in range(5)])
        iters.append(it)
    phases /= len(recs)
    ms_step = total_ms / args.steps

    # ---- end-to-end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        ch = torch.from_numpy(coeffs_h).pin_memory()
        fh = torch.from_numpy(f_h).pin_memory()
        gh = torch.from_numpy(g_h).pin_memory()
        outs = [torch.empty(x, dtype=torch.float64).pin_memory() for x in
                (g.shape, g.shape, (f.shape[0], nrhs), g.shape, coeffs.shape)]
        h2d = ch.numel() * 8 + fh.numel() * 8 + gh.numel() * 8
        d2h = sum(o.numel() * 8 for o in outs)
        # a copy stream overlaps each step's transfers with the neighbouring steps' work:
        # step k + 1's inputs are copied in while step k runs, and step k's results are
        # copied out while step k + 1 runs; the first upload and the last download are not
        # overlapped with anything
        cs = torch.cuda.Stream(device=dev)

        def upload():
            with torch.cuda.stream(cs):
                xs = [x.to(dev, non_blocking=True) for x in (ch, fh, gh)]
                e = torch.cuda.Event()
                e.record(cs)
            return xs, e

        barrier(world)
        torch.cuda.synchronize()
        e0 = ev()
        cs.wait_event(e0)
        nxt = upload()
        for k in range(args.steps):
            (cd, fd, gd), ein = nxt
            stream.wait_event(ein)
            for x in (cd, fd, gd):
                x.record_stream(stream)
            if k + 1 < args.steps:
                nxt = upload()
            res = step(cd, fd, gd, None)
            eout = torch.cuda.Event()
            eout.record(stream)
            with torch.cuda.stream(cs):
                cs.wait_event(eout)
                for o, r in zip(outs, res):
                    r.record_stream(cs)
                    o.copy_(r, non_blocking=True)
        stream.wait_stream(cs)
        e1 = ev()
        torch.cuda.synchronize()
        barrier(world)
        e2e_ms = allmax(e0.elapsed_time(e1), world) / args.steps
        e2e = {"value": world * dof / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    peaks, src = measured_peaks()
    hbm = peaks["hbm_gbs"]
    # ---- solve-only throughput at nrhs 1, 8, 64 on one built operator of each precision
    # (repeat solves: each replays its captured CUDA graph from the second call on; the
    # mixed solves run the refinement count calibrated on the first solve)
    sweep = {}
    s64 = Solver(tree, coeffs, P, "fp64", autotune=tune)
    smx = Solver(tree, coeffs, P, "mixed", autotune=tune)
    for nr in (1, 8, 64):
        fk, gk = f[:, :nr].contiguous(), g[..., :nr].contiguous()
        row = {}
        for name, s in (("fp64", s64), ("mixed", smx)):
            for _ in range(3):
                s.solve(fk, gk)
            ms, _ = timed(stream, lambda: s.solve(fk, gk), reps=5)
            ms = allmax(ms, world)
            row[name] = solve_roofline(s, nr, ms, s.last_iters, hbm)
            row[name]["dof_per_s"] *= world
            if name == "mixed":
                row[name]["ir_steps"] = s.last_iters
        sweep[str(nr)] = row
    # per-kernel record of the solves at nrhs 1 (direct launches, so that every kernel is timed)
    solve_kernels = {}
    for name, prec in (("fp64", "fp64"), ("mixed", "mixed")):
        s = Solver(tree, coeffs, P, prec, use_graphs=False, autotune=tune)
        f1, g1 = f[:, :1].contiguous(), g[..., :1].contiguous()
        for _ in range(3):
            s.solve(f1, g1)
        torch.cuda.synchronize()
        lib.hps_timing_reset()
        lib.hps_timing_enable(1)
        for _ in range(5):
            s.solve(f1, g1)
        torch.cuda.synchronize()
        lib.hps_timing_enable(0)
        tab = _native.timing_table()
        s.close()
        top = max(tab, key=lambda r: r["ms"])
        solve_kernels[name] = {
            "kernel": top["name"], "ms_per_launch": top["ms"] / max(top["launches"], 1),
            "achieved_gbs": top["bytes"] / (top["ms"] / 1e3) / 1e9,
            "hbm_frac": top["bytes"] / (top["ms"] / 1e3) / 1e9 / hbm,
            "share_of_solve": top["ms"] / sum(r["ms"] for r in tab),
            "kernels": sorted([{"name": r["name"], "launches": r["launches"] // 5, "ms": round(r["ms"] / 5, 4)}
                               for r in tab], key=lambda r: -r["ms"])[:8]}
    s64.close()
    smx.close()

    # ---- roofline of the dominant kernel of the step
    dom = max(table, key=lambda r: r["ms"])
    per_launch_ms = dom["ms"] / max(dom["launches"], 1)
    if dom["name"].startswith("gj_update_tc"):
        # the FP64 update on the tensor cores (exact digit slicing) is bound by moving the
        # updated matrix, not by arithmetic: bytes read + written per launch vs HBM
        achieved = dom["bytes"] / (dom["ms"] / 1e3) / 1e9
        roof = {"kernel": dom["name"], "bound": "hbm", "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": achieved / hbm, "peak_source": src,
                "fp64_equivalent_tflops": dom["flops"] / (dom["ms"] / 1e3) / 1e12}
    elif ("_f64" in dom["name"]) and dom["flops"] > 0:
        achieved = dom["flops"] / (dom["ms"] / 1e3) / 1e12
        roof = {"kernel": dom["name"], "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (FFMA pipe)"}
    else:
        achieved = dom["bytes"] / (dom["ms"] / 1e3) / 1e9
        roof = {"kernel": dom["name"], "bound": "hbm", "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": achieved / hbm, "peak_source": src}
    roof["traffic"] = traffic_record(dom["name"])
    roof["launches"] = dom["launches"]
    roof["ms_per_launch"] = per_launch_ms
    roof["share_of_kernel_time"] = dom["ms"] / sum(r["ms"] for r in table)
    launches = sum(r["launches"] for r in table)

    b64, s64t, a64, bm, smt = phases / 1e3
    out = {
        "metric": METRIC, "value": world * dof / (ms_step / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (mixed path: f32 sweeps + double-float residual)",
        "data": "synthetic (seeded 8-mode Fourier-series coefficients and loads)",
        "config": {"workload": workload(), "leaves": n_leaf, "p": P, "q": P - 1, "nrhs": nrhs,
                   "dof_per_rhs": n_leaf * P * P, "paper_N_per_rhs": NX * NX * (P - 1) ** 2 + 2 * NX * (P - 1) + 1,
                   "parallelism": "replicas" if world > 1 else "single",
                   "tiles": "fixed rules" if args.no_autotune else "autotuned during warm-up",
                   "l2": "inputs larger than L2 (operator store of 2.7 GB streamed per solve)"},
        "phases_s": {"build_fp64": b64, "solve_fp64": s64t, "adjoint_fp64": a64, "build_mixed": bm,
                     "solve_mixed": smt},
        "build_s": {"fp64": b64, "mixed": bm},
        "solve_dof_per_s": {"fp64": dof / s64t, "mixed": dof / smt},
        "solve_only_by_nrhs": sweep,
        "solve_kernels_nrhs1": solve_kernels,
        "grad_forward_ratio": {"adjoint_over_build_plus_solve": a64 / (b64 + s64t), "adjoint_over_solve": a64 / s64t},
        "mixed": {"rel_linf_vs_fp64": rel_err, "ir_steps": int(np.median(iters)) if iters else None},
        "gpu_launches": launches, "gpu_launches_per_step": launches / args.steps,
        "roofline": roof,
        "kernels": sorted([{"name": r["name"], "launches": round(r["launches"] / args.steps, 2),
                            "ms": round(r["ms"] / args.steps, 4)}
                           for r in table], key=lambda r: -r["ms"])[:12],
        "clocks": clk.summary(),
    }
    if e2e:
        out["e2e"] = e2e
    if not args.no_extra:
        out["workloads"] = extra_workloads(args, stream, tune, world)
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(nrhs)
    return out


# ------------------------------------------------------------------------------------
# the other workloads (outside the timed region): each reports build seconds, solve DOF/s
# and its own accuracy check

def _grid(tree, p):
    cheb = tree.nodes(p, p - 1, "cheb")
    bnd = tree.nodes(p, p - 1, "boundary")
    nl = cheb.shape[0] // (p * p)
    return cheb[:, 0].reshape(nl, p * p), cheb[:, 1].reshape(nl, p * p), bnd[:, 0], bnd[:, 1]


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float64)


def _build_timed(stream, tree, coeffs, p, prec, **kw):
    """Build twice on the same tree (the first plans, tunes and warms up) and time the
    second; returns (seconds, solver)."""
    from paper_1612_02736_gb300 import Solver
    Solver(tree, coeffs, p, prec, **kw).close()
    ms, s = timed(stream, lambda: Solver(tree, coeffs, p, prec, **kw))
    return ms / 1e3, s


def _solve_timed(stream, s, f, g, reps=3):
    for _ in range(2):
        u = s.solve(f, g)
    ms, u = timed(stream, lambda: s.solve(f, g), reps=reps)
    return ms, u


def wl_poisson(stream, tune):
    """Constant-coefficient Poisson on the unit square, 4 x 4 leaves, p = 16, with the
    manufactured solution u* = sin(pi x) sin(2 pi y) + x^2 y."""
    import synthetic as syn
    from paper_1612_02736_gb300 import Tree
    p = 16
    tree = Tree.uniform(0.0, 0.0, 1.0, 1.0, 4, 4)
    X, Y, bx, by = _grid(tree, p)
    c, g0 = syn.poisson_manufactured(X, Y)
    coeffs = _dev(np.array(c))
    ustar = syn.u_star(X, Y)
    out = {"workload": "poisson-4x4-p16", "leaves": 16, "p": p}
    for prec in ("fp64", "mixed"):
        b, s = _build_timed(stream, tree, coeffs, p, prec, autotune=tune)
        row = {"build_s": b}
        for nr in (1, 64):
            f = _dev(np.repeat(syn.u_star(bx, by)[:, None], nr, 1))
            g = _dev(np.repeat(g0[..., None], nr, 2))
            ms, u = _solve_timed(stream, s, f, g)
            row["solve_nrhs%d" % nr] = {"ms": ms, "dof_per_s": 16 * p * p * nr / (ms / 1e3)}
            row["max_err_vs_u_star"] = float(np.max(np.abs(u.cpu().numpy() - ustar[..., None])))
        s.close()
        out[prec] = row
    return out


def wl_lshape(stream, tune):
    """The L-shaped domain [-1,1]^2 minus [0,1] x [-1,0]: 32 x 32 base squares (768 leaves),
    refined 5 times toward the re-entrant corner and toward the seeded centre of a Gaussian
    point load (width 1e-3), p = 20, FP64; merges of uneven interfaces batched per level
    with autotuned tiles.  Right-hand side 1: the corner solution r^(2/3) sin(2 theta / 3)
    (harmonic, zero on the two edges at the corner) as Dirichlet data, g = 0; right-hand
    side 2: f = 0 and the point load."""
    import synthetic as syn
    from paper_1612_02736_gb300 import Tree
    p = 20
    xh = syn.lshape_load_centre()
    out = {"workload": "lshape-32x32-refined5-p20", "p": p, "load_centre": xh}
    errs = {}
    for lev in (1, 3, 5):
        tree = Tree.l_shape(16).refine([(0.0, 0.0), xh], lev)
        X, Y, bx, by = _grid(tree, p)
        nl = X.shape[0]
        coeffs = np.zeros((6, nl, p * p))
        coeffs[0] = coeffs[2] = 1.0
        coeffs = _dev(coeffs)

        def corner(x, y):
            r = np.hypot(x, y)
            th = np.mod(np.arctan2(y, x), 2 * np.pi)
            return r ** (2.0 / 3.0) * np.sin(2.0 * th / 3.0)
        f = np.stack([corner(bx, by), np.zeros_like(bx)], axis=1)
        g = np.stack([np.zeros_like(X), syn.point_load(X, Y, xh)], axis=2)
        b, s = _build_timed(stream, tree, coeffs, p, "fp64", autotune=tune)
        ms2, u = _solve_timed(stream, s, _dev(f), _dev(g))
        errs[str(lev)] = float(np.max(np.abs(u[..., 0].cpu().numpy() - corner(X, Y))))
        if lev == 5:
            f64, g64 = _dev(np.tile(f, (1, 32))), _dev(np.tile(g, (1, 1, 32)))
            ms64, _ = _solve_timed(stream, s, f64, g64)
            out.update({"leaves": nl, "build_s": b,
                        "solve_nrhs2": {"ms": ms2, "dof_per_s": nl * p * p * 2 / (ms2 / 1e3)},
                        "solve_nrhs64": {"ms": ms64, "dof_per_s": nl * p * p * 64 / (ms64 / 1e3)},
                        "point_load_max_u": float(u[..., 1].abs().max())})
        s.close()
    out["corner_solution_max_err_by_levels"] = errs
    return out


def wl_heat(stream, tune, steps):
    """Backward Euler for u_t = Laplace(u), (I - dt Laplace) u^(n+1) = u^n, dt = 1e-3, on the
    unit square with 128 x 128 leaves, p = 16 (4.2 M nodes): 64 ensemble members (sums of
    20 seeded Gaussians), Dirichlet data sin(t) x y.  One operator per precision, built
    once; the mixed stepping is compared with the FP64 stepping at steps 1, 10, 100 (and
    1000 when run that far)."""
    import torch
    import synthetic as syn
    from paper_1612_02736_gb300 import Tree
    from paper_1612_02736_gb300.heat import heat_coefficients
    n, p, dt, members = 128, 16, 1e-3, 64
    tree = Tree.uniform(0.0, 0.0, 1.0, 1.0, n, n)
    X, Y, bx, by = _grid(tree, p)
    Xd, Yd = _dev(X)[..., None], _dev(Y)[..., None]
    u0 = torch.zeros(X.shape + (members,), dtype=torch.float64, device="cuda")
    for m in range(members):  # the seeded Gaussian sums, evaluated on the device
        a, al, c = syn.heat_initial_params(member=m)
        for i in range(len(a)):
            u0[..., m:m + 1] += a[i] * torch.exp(-al[i] * ((Xd - c[i, 0]) ** 2 + (Yd - c[i, 1]) ** 2))
    bxy = _dev(bx * by)[:, None].repeat(1, members).contiguous()
    coeffs = heat_coefficients(n * n, p, dt)
    checks = [k for k in (1, 10, 100, 1000) if k <= steps]
    out = {"workload": "heat-128x128-p16", "leaves": n * n, "p": p, "dt": dt, "members": members, "steps": steps}
    ref = {}
    for prec in ("fp64", "mixed"):
        b, s = _build_timed(stream, tree, coeffs, p, prec, autotune=tune)
        u = u0
        s.solve(bxy * np.sin(dt), u)  # first call: graph capture set-up / calibration
        torch.cuda.synchronize()
        saved = {}
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for k in range(1, steps + 1):
            u = s.solve(bxy * np.sin(k * dt), u)
            if k in checks:
                saved[k] = u.clone()
        t1.record(stream)
        torch.cuda.synchronize()
        sec = t0.elapsed_time(t1) / 1e3
        row = {"build_s": b, "solve_s": sec, "ms_per_step": sec * 1e3 / steps,
               "dof_per_s": members * n * n * p * p * steps / sec, "operator_bytes": s.operator_bytes}
        if steps < 1000:
            row["solve_s_1000_steps_extrapolated"] = sec * 1000.0 / steps
        if prec == "fp64":
            ref = saved
        else:
            row["ir_steps_last"] = s.last_iters
            row["rel_linf_vs_fp64_by_step"] = {str(k): float((saved[k] - ref[k]).abs().max() / ref[k].abs().max())
                                               for k in checks}
        s.close()
        out[prec] = row
    del ref
    torch.cuda.empty_cache()
    return out


def wl_adjoint_recompute(stream):
    """Adjoint gradient of J = 0.5 ||u - u_obs||^2 over all collocation nodes with respect
    to the coefficient fields (c among them) and the load, for the variable-coefficient
    operator at 64 x 64 leaves, p = 16, through the autograd function with leaf operators
    recomputed in the backward pass (store_leaf_ops = False), and with stored operators.
    u_obs is the solution at the perturbed c.  The gradient is checked by central finite
    differences (h = 1e-6) along 10 seeded smooth directions of c."""
    import torch
    import synthetic as syn
    from paper_1612_02736_gb300 import Solver, Tree
    from paper_1612_02736_gb300.solver import HPSFunction
    p = 16
    tree = Tree.uniform(0.0, 0.0, 1.0, 1.0, 64, 64)
    coeffs_h, cobs_h, f_h, g_h = make_inputs(tree, 1)
    f, g = _dev(f_h[:, 0]), _dev(g_h[..., 0])
    s = Solver(tree, _dev(cobs_h), p, "fp64")
    u_obs = s.solve(f, g)
    s.close()
    out = {"workload": "adjoint-varcoef-64x64-p16"}

    def J_of(c, store):
        u = HPSFunction.apply(c, f, g, tree, p, store)
        return 0.5 * ((u - u_obs) ** 2).sum()

    grads = {}
    for store in (False, True):
        c = _dev(coeffs_h).requires_grad_(True)
        J_of(c, store).backward()  # warm-up
        c.grad = None
        fwd, J = timed(stream, lambda: J_of(c, store))
        bwd, _ = timed(stream, lambda: J.backward())
        out["recompute" if not store else "stored"] = {"forward_ms": fwd, "backward_ms": bwd,
                                                       "grad_over_forward": bwd / fwd}
        grads[store] = c.grad.detach().clone()
    grad = grads[True]
    out["recompute_vs_stored_grad_rel_linf"] = float((grads[False] - grad).abs().max() / grad.abs().max())
    # central differences along 10 seeded smooth directions of c, each scaled to unit
    # max-norm: at the specified h = 1e-6 the quotient carries the rounding of the two solves
    # divided by h; at h = 1e-3 that noise is a thousand times smaller (truncation ~1e-6)
    X, Y, _, _ = _grid(tree, p)
    errs = {1e-6: [], 1e-3: []}
    for v1 in syn.smooth_directions(X, Y, n=10, seed_offset=1100, fields=1):
        v = _dev(v1[0] / np.abs(v1[0]).max())
        ad = float((grad[5] * v).sum())
        for h in errs:
            with torch.no_grad():
                cp, cm = _dev(coeffs_h), _dev(coeffs_h)
                cp[5] += h * v
                cm[5] -= h * v
                jp, jm = J_of(cp, True).item(), J_of(cm, True).item()
            errs[h].append(abs((jp - jm) / (2 * h) - ad) / max(abs(ad), 1e-300))
    checks = {"directions": 10}
    for h, e in errs.items():
        checks["h=%g" % h] = {"max_rel_err": max(e), "rel_errs": e}
    out["fd_check_c"] = checks
    return out


def wl_p_sweep(stream, tune):
    """The variable-coefficient workload at 64 x 64 leaves for p = 16, 20, 24, 30: build
    seconds and solve DOF/s in FP64 and mixed precision."""
    import torch
    from paper_1612_02736_gb300 import Tree
    tree = Tree.uniform(0.0, 0.0, 1.0, 1.0, 64, 64)
    out = {}
    for p in (16, 20, 24, 30):
        coeffs_h, _, f_h, g_h = make_inputs(tree, 64, p=p)
        coeffs = _dev(coeffs_h)
        row = {}
        for prec in ("fp64", "mixed"):
            b, s = _build_timed(stream, tree, coeffs, p, prec, autotune=tune)
            r = {"build_s": b, "operator_bytes": s.operator_bytes}
            for nr in (1, 64):
                f, g = _dev(f_h[:, :nr]), _dev(g_h[..., :nr])
                ms, _ = _solve_timed(stream, s, f, g, reps=2)
                r["solve_nrhs%d" % nr] = {"ms": ms, "dof_per_s": 4096 * p * p * nr / (ms / 1e3)}
                if prec == "mixed":
                    r["ir_steps_nrhs%d" % nr] = s.last_iters
            s.close()
            row[prec] = r
        out[str(p)] = row
        del coeffs
        torch.cuda.empty_cache()
    return out


def extra_workloads(args, stream, tune, world):
    import torch
    out = {}
    for name, fn in (("poisson_4x4_p16", lambda: wl_poisson(stream, tune)),
                     ("lshape_refined_p20", lambda: wl_lshape(stream, tune)),
                     ("heat_128x128_p16", lambda: wl_heat(stream, tune, args.heat_steps)),
                     ("adjoint_recompute_64x64_p16", lambda: wl_adjoint_recompute(stream)),
                     ("p_sweep_64x64", lambda: wl_p_sweep(stream, tune))):
        t0 = time.perf_counter()
        out[name] = fn()
        out[name]["wall_s"] = time.perf_counter() - t0
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------------------------
# CPU oracle: FP64 build + solve + adjoint (+ coefficient gradients) per step on an n x n
# leaf sub-square of the workload (leaf size 1/64; n = 64 is the whole workload)

def oracle_step(n, nrhs):
    import synthetic as syn
    from oracle import hps, tree as tr
    from oracle.points import boundary_points, leaf_points
    side = n / 64
    t = tr.uniform_tree(0.0, 0.0, side, side, n, n, P - 1)
    X, Y = leaf_points(t, P)
    bx, by = boundary_points(t)
    prob = syn.VarCoeffProblem()
    coeffs = np.array(prob.coeffs(X, Y))
    scale = np.linspace(0.5, 1.5, nrhs)
    g = prob.load(X, Y)[..., None] * scale
    f = prob.dirichlet(bx, by)[:, None] * scale
    t0 = time.perf_counter()
    ops = hps.build(t, coeffs, P)
    u, _ = hps.solve(t, ops, P, f, g)
    _, gb, _ = hps.adjoint(t, ops, P, u)
    hps.coeff_gradients(t, P, u, gb)
    return time.perf_counter() - t0, t.n_leaves * P * P * nrhs


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return max(n)
    except Exception:
        pass
    return int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))


def cpu_baseline(nrhs):
    dt, dof = oracle_step(64, nrhs)
    return {"value": dof / dt, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
            "sample": "the whole workload once (64x64 leaves, p=16, nrhs=%d): FP64 build + solve + adjoint "
                      "+ coefficient gradients, %.1f s; BLAS threads = host cores" % (nrhs, dt),
            "seconds": dt}


REF_N = 16  # leaves per side of the reference arm's sample


def run_reference(args, rank, world):
    if rank != 0:
        return None
    nrhs = args.nrhs
    for _ in range(args.warmup):
        oracle_step(REF_N, nrhs)
    times, dofs = [], 0
    for _ in range(args.steps):
        dt, dof = oracle_step(REF_N, nrhs)
        times.append(dt)
        dofs = dof
    ms = 1e3 * float(np.mean(times))
    val = dofs / (ms / 1e3)
    sample = ("%dx%d leaves of the workload (sub-square [0,%g]^2, leaf size 1/64, p=16, nrhs=%d) per step: "
              "FP64 build + solve + adjoint + coefficient gradients" % (REF_N, REF_N, REF_N / 64, nrhs))
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "varcoef-%dx%d-p16 (sample of varcoef-64x64-p16)" % (REF_N, REF_N),
                       "leaves": REF_N * REF_N, "p": P, "q": P - 1, "nrhs": nrhs},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_gpu(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
