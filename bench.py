#!/usr/bin/env python3
"""Benchmark of the GB300 HPS solver on the variable-coefficient workload: 64 x 64 leaves,
p = 16 (q = 15), seeded 8-mode Fourier-series coefficients, a batch of nrhs right-hand
sides.

One step is one pass of the whole hot path over one batch:
  FP64 build (leaf eliminations + merges), FP64 solve of the batch, the adjoint of the
  batch (gradients of J = 0.5 ||u - u_obs||^2 w.r.t. f, g and the six coefficient
  fields), then the mixed-precision build and the mixed solve (FP32 sweeps refined
  against FP64 residuals to max|du| <= 1e-10 max|u|).
value = solved degrees of freedom (leaf-major n_leaf p^2 per right-hand side) per second
of step time, whole job.  Phase timings give build seconds, solve DOF/s (FP64 vs mixed)
and the gradient/forward ratio.

--impl reference times the CPU oracle (FP64 NumPy restatement of the method) on a bounded
sample of the same workload instead.  Launch with torchrun for several GPUs: every rank
solves its own replica (no data-path collective).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = 64
P = 16
METRIC = "build s & solve DOF/s at 1e-8 rel err: mixed vs FP64 GPU; grad/forward ratio"
UNIT = "DOF/s"
# FP64 FFMA peak of GB300: 152 SMs x 2 FP64 FMA/clock/SM x 2 flop x 2070 MHz (the 1.25
# TFLOP/s FP64 figure at the maximum SM clock); no FP64 tensor path is faster on this part.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--nrhs", type=int, default=64)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
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
        barrier(world)
        torch.cuda.synchronize()
        e0 = ev()
        for _ in range(args.steps):
            cd = ch.to(dev, non_blocking=True)
            fd = fh.to(dev, non_blocking=True)
            gd = gh.to(dev, non_blocking=True)
            res = step(cd, fd, gd, None)
            for o, r in zip(outs, res):
                o.copy_(r, non_blocking=True)
        e1 = ev()
        torch.cuda.synchronize()
        barrier(world)
        e2e_ms = allmax(e0.elapsed_time(e1), world) / args.steps
        e2e = {"value": world * dof / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---- solve-only throughput at nrhs 1, 8, 64 on one built operator of each precision
    # (repeat solves: the FP64 sweep replays its captured CUDA graph from the second call)
    sweep = {}
    s64 = Solver(tree, coeffs, P, "fp64", autotune=tune)
    smx = Solver(tree, coeffs, P, "mixed", autotune=tune)
    for nr in (1, 8, 64):
        fk, gk = f[:, :nr].contiguous(), g[..., :nr].contiguous()
        row = {}
        for name, s in (("fp64", s64), ("mixed", smx)):
            for _ in range(3):
                s.solve(fk, gk)
            torch.cuda.synchronize()
            a = ev()
            for _ in range(5):
                s.solve(fk, gk)
            b = ev()
            torch.cuda.synchronize()
            ms = allmax(a.elapsed_time(b), world) / 5
            row[name] = {"ms": ms, "dof_per_s": world * n_leaf * P * P * nr / (ms / 1e3)}
        sweep[str(nr)] = row
    s64.close()
    smx.close()

    # ---- roofline of the dominant kernel
    peaks, src = measured_peaks()
    dom = max(table, key=lambda r: r["ms"])
    per_launch_ms = dom["ms"] / max(dom["launches"], 1)
    if dom["name"].startswith("gj_update_tc"):
        # the FP64 update on the tensor cores (exact digit slicing) is bound by moving the
        # updated matrix, not by arithmetic: bytes read + written per launch vs HBM
        achieved = dom["bytes"] / (dom["ms"] / 1e3) / 1e9
        roof = {"kernel": dom["name"], "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "peak_source": src,
                "fp64_equivalent_tflops": dom["flops"] / (dom["ms"] / 1e3) / 1e12}
    elif ("_f64" in dom["name"]) and dom["flops"] > 0:
        achieved = dom["flops"] / (dom["ms"] / 1e3) / 1e12
        roof = {"kernel": dom["name"], "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (FFMA pipe)"}
    else:
        achieved = dom["bytes"] / (dom["ms"] / 1e3) / 1e9
        roof = {"kernel": dom["name"], "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "peak_source": src}
    traf = traffic_record(dom["name"])
    roof["traffic"] = traf
    roof["launches"] = dom["launches"]
    roof["ms_per_launch"] = per_launch_ms
    roof["share_of_kernel_time"] = dom["ms"] / sum(r["ms"] for r in table)
    launches = sum(r["launches"] for r in table)

    b64, s64, a64, bm, sm = phases / 1e3
    out = {
        "metric": METRIC, "value": world * dof / (ms_step / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (mixed path: f32 sweeps + f64 residual)",
        "data": "synthetic (seeded 8-mode Fourier-series coefficients and loads)",
        "config": {"workload": workload(), "leaves": n_leaf, "p": P, "q": P - 1, "nrhs": nrhs,
                   "dof_per_rhs": n_leaf * P * P, "paper_N_per_rhs": NX * NX * (P - 1) ** 2 + 2 * NX * (P - 1) + 1,
                   "parallelism": "replicas" if world > 1 else "single",
                   "tiles": "fixed rules" if args.no_autotune else "autotuned during warm-up",
                   "l2": "inputs larger than L2 (operator store of 2.7 GB streamed per solve)"},
        "phases_s": {"build_fp64": b64, "solve_fp64": s64, "adjoint_fp64": a64, "build_mixed": bm,
                     "solve_mixed": sm},
        "build_s": {"fp64": b64, "mixed": bm},
        "solve_dof_per_s": {"fp64": dof / s64, "mixed": dof / sm},
        "solve_only_by_nrhs": sweep,
        "grad_forward_ratio": {"adjoint_over_build_plus_solve": a64 / (b64 + s64), "adjoint_over_solve": a64 / s64},
        "mixed": {"rel_linf_vs_fp64": rel_err, "ir_steps": int(np.median(iters)) if iters else None},
        "gpu_launches": launches, "gpu_launches_per_step": launches / args.steps,
        "roofline": roof,
        "kernels": sorted([{"name": r["name"], "launches": r["launches"], "ms": round(r["ms"] / args.steps, 4)}
                           for r in table], key=lambda r: -r["ms"])[:12],
        "clocks": clk.summary(),
    }
    if e2e:
        out["e2e"] = e2e
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(nrhs, sample_n=32)
    return out


# ------------------------------------------------------------------------------------
# CPU oracle: a bounded sample of the workload (16 x 16 leaves of the same 1/64 leaf size,
# i.e. the sub-square [0, 1/4]^2), FP64 build + solve + adjoint per step.

def oracle_step(sample_n, nrhs):
    import synthetic as syn
    from oracle import hps, tree as tr
    from tests.helpers import boundary_points, leaf_points
    side = sample_n / NX
    t = tr.uniform_tree(0.0, 0.0, side, side, sample_n, sample_n, P - 1)
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
    return os.cpu_count()


def cpu_baseline(nrhs, sample_n=32):
    dt, dof = oracle_step(sample_n, nrhs)
    return {"value": dof / dt, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
            "sample": "%dx%d leaves of the same workload (sub-square [0,%g]^2, leaf size 1/64, p=16, nrhs=%d): "
                      "FP64 build + solve + adjoint, %.1f s" % (sample_n, sample_n, sample_n / NX, nrhs, dt),
            "seconds": dt}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    nrhs = args.nrhs
    for _ in range(args.warmup):
        oracle_step(16, nrhs)
    times, dofs = [], 0
    for _ in range(args.steps):
        dt, dof = oracle_step(16, nrhs)
        times.append(dt)
        dofs = dof
    ms = 1e3 * float(np.mean(times))
    val = dofs / (ms / 1e3)
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload(), "leaves": NX * NX, "p": P, "q": P - 1, "nrhs": nrhs},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                             "sample": "16x16 leaves of the same workload (sub-square [0,1/4]^2, leaf size 1/64, "
                                       "p=16, nrhs=%d) per step: FP64 build + solve + adjoint" % nrhs},
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
