#!/usr/bin/env python3
"""Benchmark of the 3D Laplace FMM mat-vec on GB300.

Workload: N = 4,194,304 Plummer-sphere points (scale 1, radii <= 10), equal
charges 1/N, expansion order p = 8, mixed precision (FP32 P2P/M2L, FP64
coarse M2M/L2L, compensated per-target totals), leaf size autotuned.  One
step = one pass of the whole hot path, forward and adjoint, as a training
step runs it: root cube + Morton keys + radix sort + octree + U/V/W/X lists
(fmm_plan_rebuild), the mat-vec P2M/M2M/M2L/P2L/L2L/L2P/M2P/P2P + reduction
for phi and grad phi (fmm_eval), and the adjoint of L = sum w_i phi_i with
the forward gradient stored (fmm_adjoint: dL/dq and dL/dx, one more mat-vec).

value      = N x ranks / (max over ranks of the mean device time per step)
e2e        = the same step through fmm_solve_adjoint_host on pinned HOST
             buffers, the H2D copy of points, charges and weights and the D2H
             copy of phi, grad, dL/dq and dL/dx inside every timed step
roofline   = the dominant pass, from CUDA events the library records on its
             stream during the timed steps, against the FP32 rate measured on
             this GPU by fmm_fp32_peak
cpu_baseline = the CPU oracle (plain C, FP64, OpenMP) on the same N = 4M
             points at the same leaf size, forward and adjoint; the same leg
             evaluates the oracle's direct sum at 4096 sampled targets, the
             reference of the error statement

`--impl reference` times the oracle itself as the reference arm.
Multi-GPU (torchrun): replicas only -- every rank solves its own problem,
no collective on the data path.
"""
import argparse
import ctypes
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "3D Laplace FMM evals/s at N=4M at stated rel. error; fwd+adjoint vs plain FP64"
UNIT = "evals/s"
PASSES = ["keys+sort", "boxes", "lists", "P2M", "M2M", "M2L", "P2L", "L2L", "L2P", "M2P", "P2P",
          "reduce"]
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM (Blackwell)

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernel, from one ncu capture of the same kernel and workload, keyed
# by (pass, N, order, leaf size, precision, staging shape); any other
# configuration, or a
# kernel changed since the capture, reports null.
TRAFFIC_BYTES = {
    # k_p2p_f32<160, 2, 16>, leaves by work class; the lists as defined (no direct W/X pairs)
    ("P2P", 4194304, 8, 128, "mixed", 1, False): 944.61e6,
    # the same kernel with the W/X pairs of small leaves in the U lists (the default)
    ("P2P", 4194304, 8, 128, "mixed", 1, True): 990.00e6,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=4194304)
    ap.add_argument("--order", type=int, default=8)
    ap.add_argument("--leaf", type=int, default=0, help="leaf size; 0 = autotune (default)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--m2l-path", default="auto", choices=["auto", "simt", "tensor"],
                    help="M2L engine of the mixed path: auto (tensor cores), simt (FP32 CUDA "
                         "cores), tensor")
    ap.add_argument("--p2p-tile", type=int, default=0,
                    help="staging shape of the FP32 near-field kernel (0 = default)")
    ap.add_argument("--m2l-tile", type=int, default=0,
                    help="operand form of the tensor-core M2L: 1 TF32, 2 FP16 (0 = default)")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="points in the oracle's CPU-baseline run (0 = the full N)")
    ap.add_argument("--ref-sample", type=int, default=524288,
                    help="points per step of the reference arm (the CPU oracle)")
    ap.add_argument("--ref-leaf", type=int, default=128,
                    help="leaf size of the reference arm (the GPU autotuner's choice for the "
                         "4M Plummer workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 comparison leg")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 256-problem leg")
    ap.add_argument("--batch-leaf", type=int, default=0,
                    help="leaf size of the batched leg; 0 = autotune (default)")
    ap.add_argument("--dual-theta", type=float, default=0.75,
                    help="also time the dual-tree walk (acceptance theta) on the same points; 0 skips")
    ap.add_argument("--precond", action="store_true",
                    help="add the FMM-preconditioned solves of the 7-point Laplace (CG) and "
                         "Helmholtz (flexible GMRES) problems")
    ap.add_argument("--wx-direct", default="on", choices=["on", "off"],
                    help="W/X pairs of two leaves whose W leaf holds at most (p+1)^2 points by the "
                         "direct sum (fmm_opts.wx_direct; on by default), or the lists as defined")
    ap.add_argument("--no-helmholtz", action="store_true",
                    help="skip the Helmholtz mat-vec (kappa = 7) on the h = 2^-5 grid of [-1,1]^3")
    ap.add_argument("--no-lattice", action="store_true",
                    help="skip plan/eval time and peak device memory vs N on uniform lattices")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the raw samples; FMM_BENCH_CLOCKS_DIR keeps them, else a temporary directory
        self.path = os.path.join(os.environ.get("FMM_BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 "fmm_bench_clocks_rank%d.csv" % index)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ oracle
def cpu_baseline(n_sample, order, leaf, sel, n_one_core=131072, direct_wx=0):
    """The CPU oracle (FP64 plan + FMM with gradients, forward and adjoint: an
    evaluation with the charges and one with the loss weights) on the Plummer
    points of the benchmark (all of them when n_sample is the full N), on all
    host cores, and on one core (a subprocess with OMP_NUM_THREADS=1) on a
    smaller sample.  Also returns the oracle's FP64 direct sum (phi, grad) at
    the sampled targets `sel`, the reference of the error statement."""
    import oracle
    from paper_1602_02244_gb300 import workloads
    xyz, q = workloads.plummer_problem(n_sample, 0)
    w = workloads.rng(2).normal(size=n_sample)
    t0 = time.perf_counter()
    tree = oracle.Tree(xyz, leaf, direct_wx=direct_wx)
    tree.eval(order, q, grad=True)
    tree.eval(order, w, grad=True)
    dt = time.perf_counter() - t0
    del tree
    out = {"value": n_sample / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": "Plummer N=%d (the benchmark's points, charges 1/N), p=%d, leaf %d%s: plan + "
                     "FP64 FMM forward (phi, grad) + adjoint (the FMM with the loss weights), "
                     "%.1f s" % (n_sample, order, leaf,
                                 ", the same direct W/X leaf pairs" if direct_wx else "", dt)}
    code = ("import json, time, oracle\n"
            "from paper_1602_02244_gb300 import workloads\n"
            "xyz, q = workloads.plummer_problem(%d, 0)\n"
            "w = workloads.rng(2).normal(size=%d)\n"
            "t0 = time.perf_counter()\n"
            "t = oracle.Tree(xyz, %d, direct_wx=%d)\n"
            "t.eval(%d, q, grad=True)\n"
            "t.eval(%d, w, grad=True)\n"
            "print(json.dumps({'s': time.perf_counter() - t0, 'cores': oracle.num_threads()}))\n"
            % (n_one_core, n_one_core, leaf, direct_wx, order, order))
    try:
        env = dict(os.environ, OMP_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                           text=True, timeout=300)
        one = json.loads(r.stdout.strip().splitlines()[-1])
        out["one_core"] = {"value": n_one_core / one["s"], "unit": UNIT, "cores": one["cores"],
                           "sample": "Plummer N=%d, same order, leaf and step, %.1f s"
                                     % (n_one_core, one["s"])}
    except Exception as e:  # reported, not fatal
        out["one_core"] = {"error": str(e)[:200]}
    t0 = time.perf_counter()
    ref = oracle.direct(xyz, q, xyz[sel])
    out["direct_s"] = time.perf_counter() - t0
    return out, ref


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1602_02244_gb300 import workloads
    n = args.ref_sample
    leaf = args.leaf or args.ref_leaf
    xyz, q = workloads.plummer_problem(n, 0)
    w = workloads.rng(2).normal(size=n)

    direct_wx = (args.order + 1) ** 2 if args.wx_direct == "on" else 0

    def step():
        t = oracle.Tree(xyz, leaf, direct_wx=direct_wx)
        t.eval(args.order, q, grad=True)
        t.eval(args.order, w, grad=True)

    for _ in range(min(args.warmup, 1)):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    val = n / (ms / 1e3)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "Plummer N=%d per step (bounded CPU sample of the N=4,194,304 "
                                   "problem), p=%d, leaf %d, FP64%s; step = plan + forward "
                                   "(phi, grad) + adjoint (the FMM with the loss weights)"
                                   % (n, args.order, leaf,
                                      ", W/X pairs of small leaves direct" if direct_wx else "")},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": "Plummer N=%d per step: plan + FP64 FMM forward + adjoint, "
                                       "leaf %d" % (n, leaf)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- ours
def max_over_ranks(value, world, device=None):
    """Largest `value` over all ranks (the slowest replica sets the step time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def algorithmic_work(plan):
    """Per-step algorithmic work from the plan layout: P2P pairs (targets x
    U-list sources) and M2L matvecs (|V| pairs)."""
    e = plan.export()
    cnt = e["box_count"].astype(np.int64)
    u_off, u_idx = e["u_off"], e["u_idx"]
    src_per_leaf = np.add.reduceat(cnt[u_idx], u_off[:-1]) if len(u_idx) else np.zeros(0)
    rows = np.diff(u_off)
    src = np.where(rows > 0, src_per_leaf, 0)
    pairs = int(np.sum(cnt * src))
    v_pairs = int(len(e["v_idx"]))
    return pairs, v_pairs, e


def batched_leg(dev, steps, warmup, leaf=0, wx_direct=False):
    """256 independent uniform problems, N log-uniform in [2048, 65536], p = 6,
    mixed precision, leaf size `leaf` (0: autotuned): forward (phi, grad) plus
    adjoint (dL/dq, dL/dx) replayed as one CUDA graph per step."""
    import torch
    from paper_1602_02244_gb300 import binding, workloads
    sizes, pts, qs = workloads.batch_problem(256, 0)
    off = np.concatenate([[0], np.cumsum(sizes)])
    total = int(off[-1])
    X = torch.tensor(np.vstack(pts), device=dev)
    Q = torch.tensor(np.concatenate(qs), device=dev)
    W = torch.tensor(workloads.rng(2).normal(size=total), device=dev)
    plan = binding.Plan(X, leaf_size=leaf, order=6, precision="mixed", offsets=off,
                        wx_direct=wx_direct)
    s = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(s):
        phi = torch.empty(total, dtype=torch.float64, device=dev)
        g = torch.empty(total, 3, dtype=torch.float64, device=dev)
        dq = torch.empty_like(phi)
        dx = torch.empty_like(g)
        for _ in range(max(warmup, 3)):
            plan.eval_graph(Q, phi, g, W, dq, dx)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        s.synchronize()
        e0.record(s)
        for _ in range(steps):
            plan.eval_graph(Q, phi, g, W, dq, dx)
        e1.record(s)
        e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    leaf = plan.sizes()["leaf_size"]
    plan.close()
    return {"problems": 256, "points": total, "leaf": leaf, "value": total / (ms / 1e3),
            "unit": "evals/s", "ms": ms,
            "mode": "p=6 mixed; forward (phi, grad) + adjoint (dL/dq, dL/dx) as one CUDA graph "
                    "launch per step over all 256 problems"}


def lattice_leg(dev, order=8):
    """The paper's FMM workload (§4.1): uniform lattices of growing N, time of
    the precalculation (plan) and of the mat-vec (eval), and the peak device
    memory of the plan, all in FP64 and mixed precision."""
    import torch
    from paper_1602_02244_gb300 import binding
    L = binding.library()
    L.fmm_memory_usage.argtypes = [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                   ctypes.c_int]
    rows = []
    from paper_1602_02244_gb300 import workloads
    for side in (16, 32, 64, 128, 160):
        xyz = workloads.lattice(side)
        n = len(xyz)
        X = torch.tensor(xyz, device=dev)
        Q = torch.ones(n, dtype=torch.float64, device=dev)
        for prec in ("mixed", "fp64"):
            torch.cuda.synchronize()
            cur, peak = ctypes.c_uint64(), ctypes.c_uint64()
            L.fmm_memory_usage(ctypes.byref(cur), ctypes.byref(peak), 1)
            base = cur.value
            t0 = time.perf_counter()
            plan = binding.Plan(X, leaf_size=64, order=order, precision=prec)
            plan.eval(Q)  # operators and workspace
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.rebuild(X)
            e1.record()
            e1.synchronize()
            t_plan = e0.elapsed_time(e1)
            e0.record()
            plan.eval(Q)
            e1.record()
            e1.synchronize()
            t_eval = e0.elapsed_time(e1)
            L.fmm_memory_usage(ctypes.byref(cur), ctypes.byref(peak), 0)
            rows.append({"n": n, "precision": prec, "plan_ms": t_plan, "eval_ms": t_eval,
                         "peak_bytes": int(peak.value - base),
                         "bytes_per_point": (peak.value - base) / n})
            plan.close()
    return rows


def precond_leg(dev, h=2.0 ** -5, tol=1e-8):
    """The paper's preconditioning experiment (§4.2), Laplace part: -Laplace u = 1
    on [-1, 1]^3, u = 0 on the boundary, 7-point stencil at spacing h; CG
    iterations and solve time without a preconditioner and with the FMM
    (free-space Green's function, mixed precision) at low orders."""
    import torch
    from paper_1602_02244_gb300 import binding, precond
    m = int(round(2.0 / h)) - 1
    b = torch.ones(m ** 3, dtype=torch.float64, device=dev)
    A = lambda v: binding.laplace7(v, h)
    precond.fpcg(A, b, None, tol=tol, maxiter=3)  # first-call initialisation, untimed
    rows = []
    for order in (None, 2, 3, 4):
        pre = precond.GreenPreconditioner(h, order=order, leaf_size=64, device=dev) if order else None
        if pre is not None:
            pre(b)  # operators and workspace
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, it, hist = precond.fpcg(A, b, pre, tol=tol, maxiter=2000)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        row = {"preconditioner": "FMM p=%d" % order if order else "none", "iterations": it,
               "rel_residual": hist[-1], "solve_ms": 1e3 * dt}
        if pre is not None:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                pre(b)
            e1.record()
            e1.synchronize()
            row["apply_ms"] = e0.elapsed_time(e1) / 5
            pre.close()
        rows.append(row)
    return {"problem": "-Laplace u = 1 on [-1,1]^3, u = 0 on the boundary, 7-point stencil, "
                       "h = 2^-5 (%d unknowns), CG to relative residual %.0e" % (m ** 3, tol),
            "runs": rows}


def helmholtz_precond_rows(dev, h=2.0 ** -5, kappa=7.0, tol=1e-8):
    """The Helmholtz half of §4.2 (Fig. 6): -Laplace u - kappa^2 u = 1 on [-1,1]^3,
    u = 0 on the boundary, h = 2^-5, kappa = 7; restarted flexible GMRES(50)
    without a preconditioner and with the Helmholtz FMM (real part of the
    outgoing Green's function, near field in FP32) at low orders."""
    import torch
    from paper_1602_02244_gb300 import binding, precond
    m = int(round(2.0 / h)) - 1
    b = torch.ones(m ** 3, dtype=torch.float64, device=dev)
    A = lambda v: binding.helmholtz7(v, h, kappa)
    precond.fgmres(A, b, None, tol=tol, maxiter=3)  # first-call initialisation, untimed
    rows = []
    for order in (None, 2, 3, 4, 6):
        pre = precond.HelmholtzGreenPreconditioner(h, kappa, order=order, leaf_size=64,
                                                   device=dev) if order else None
        if pre is not None:
            pre(b)  # operators and workspace
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, it, hist = precond.fgmres(A, b, pre, tol=tol, restart=50, maxiter=3000)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        row = {"preconditioner": "Helmholtz FMM p=%d" % order if order else "none",
               "iterations": it, "rel_residual": hist[-1], "solve_ms": 1e3 * dt}
        if pre is not None:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                pre(b)
            e1.record()
            e1.synchronize()
            row["apply_ms"] = e0.elapsed_time(e1) / 5
            pre.close()
        rows.append(row)
    return {"problem": "-Laplace u - %g^2 u = 1 on [-1,1]^3, u = 0 on the boundary, 7-point "
                       "stencil, h = 2^-5 (%d unknowns), flexible GMRES(50) to relative residual "
                       "%.0e" % (kappa, m ** 3, tol), "runs": rows}


def helmholtz_leg(dev, L, steps=5, kappa=7.0, h=2.0 ** -5, leaf=64):
    """The Helmholtz mat-vec (kernel e^{i kappa r}/r, §1 and §4.2) on the
    paper's Helmholtz domain: the h = 2^-5 interior grid of [-1,1]^3 (63^3 =
    250,047 points), kappa = 7, complex charges U[-1,1] + i U[-1,1].  Per
    precision and order: mat-vec time (CUDA events over `steps` calls,
    operators built before), per-pass times, and the roofline of M2L (8 flop
    per complex multiply-add, (p+1)^4 per V pair) against the measured FP64
    rate (FP64 plans) or FP32 rate (mixed plans, whose M2L runs in FP32).  cpu_baseline: the oracle's FP64
    direct sum at 256 sampled targets, against which each run's error is
    stated."""
    import ctypes
    import numpy as np
    import torch
    from paper_1602_02244_gb300 import binding, precond, workloads
    pts, m = precond.grid_points(h, device=dev)
    n = m ** 3
    g = workloads.rng(21)
    q_h = g.uniform(-1, 1, n) + 1j * g.uniform(-1, 1, n)
    q = torch.tensor(q_h, device=dev)
    fp64_tf = binding.fp64_peak()
    fp32_tf = binding.fp32_peak()
    sel = workloads.sample_targets(n, 256, seed=3)
    cpu = None
    xyz_h = pts.cpu().numpy()
    runs = []
    names = ["sort", "boxes", "lists", "P2M", "M2M", "M2L", "P2L", "L2L", "L2P", "M2P", "P2P",
             "reduce"]
    for precision in ("fp64", "mixed"):
        plan = binding.Plan(pts, leaf_size=leaf, order=4, precision=precision)
        ex = plan.export()
        cnt = ex["box_count"].astype(np.int64)
        uo, ui = ex["u_off"], ex["u_idx"]
        leaves = np.nonzero(ex["box_nchild"] == 0)[0]
        p2p_pairs = int(sum(cnt[b] * cnt[ui[uo[b]:uo[b + 1]]].sum() for b in leaves))
        nv = int(plan.sizes()["nv"])
        for order in (4, 8):
            phi = plan.helmholtz(q, kappa, order)
            for _ in range(2):
                plan.helmholtz(q, kappa, order, out=phi)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(steps):
                plan.helmholtz(q, kappa, order, out=phi)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
            ma = (ctypes.c_double * 12)()
            la = (ctypes.c_int64 * 12)()
            L.fmm_profile(plan._h, 1)
            L.fmm_profile_read(plan._h, ma, la)
            plan.helmholtz(q, kappa, order, out=phi)
            torch.cuda.synchronize()
            L.fmm_profile_read(plan._h, ma, la)
            L.fmm_profile(plan._h, 0)
            passes = {names[i]: ma[i] for i in range(12) if ma[i] > 0}
            if cpu is None:
                import oracle
                t0 = time.perf_counter()
                ref = oracle.h_direct(xyz_h, q_h, kappa, xyz_h[sel])
                dt = time.perf_counter() - t0
                cpu = {"value": len(sel) * n / dt, "unit": "pair interactions/s",
                       "cores": oracle.num_threads(), "kind": "oracle",
                       "sample": "FP64 direct sum at %d sampled targets over all %d sources"
                                 % (len(sel), n)}
            got = phi.cpu().numpy()[sel]
            nc = (order + 1) ** 2
            m2l_flop = 8.0 * nc * nc * nv
            peak = fp64_tf if precision == "fp64" else fp32_tf
            row = {"precision": precision, "order": order, "ms": ms,
                   "value": n / (ms / 1e3), "unit": "targets/s",
                   "rel_error_vs_oracle_direct": float(np.linalg.norm(got - ref) /
                                                       np.linalg.norm(ref)),
                   "passes_ms": passes, "v_pairs": nv, "p2p_pairs": p2p_pairs,
                   "m2l_roofline": {"bound": "alu", "achieved": m2l_flop / (passes["M2L"] / 1e3) / 1e12,
                                    "peak": peak, "unit": "TFLOP/s",
                                    "frac": m2l_flop / (passes["M2L"] / 1e3) / 1e12 / peak,
                                    "peak_source": ("fmm_fp64_peak, FP64 FMA chains (of measured)"
                                                    if precision == "fp64" else
                                                    "fmm_fp32_peak, paired FP32 FMA chains (of "
                                                    "measured): the mixed M2L runs in FP32")}}
            runs.append(row)
        plan.close()
    return {"workload": "Helmholtz e^{i 7 r}/r mat-vec, interior grid of [-1,1]^3 at h = 2^-5 "
                        "(%d points), leaf %d" % (n, leaf), "kappa": kappa,
            "fp64_peak_tflops": fp64_tf, "fp32_peak_tflops": fp32_tf, "runs": runs,
            "cpu_baseline": cpu}


def dual_leg(X, Q, S, p, precision, theta, rel_err, steps, stream, ms_lists, ms_eval_lists):
    """The same points and order with the dual-tree walk (§2.1: Dehnen's walk
    with acceptance r_T + r_S < theta |c_T - c_S|) instead of the U/V/W/X
    lists: plan + eval and eval-only time, error on the same sampled targets,
    pair counts and per-pass times."""
    import torch
    from paper_1602_02244_gb300 import binding
    L = binding.library()
    plan = binding.Plan(X, leaf_size=S, order=p, precision=precision, interaction="dual",
                        theta=theta)
    phi, g = plan.eval(Q)
    err = rel_err(phi, g)
    plan.rebuild(X)
    plan.eval(Q, out=(phi, g))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        plan.rebuild(X)
        plan.eval(Q, out=(phi, g))
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    e0.record(stream)
    for _ in range(steps):
        plan.eval(Q, out=(phi, g))
    e1.record(stream)
    e1.synchronize()
    ms_eval = e0.elapsed_time(e1) / steps
    ms_arr = (ctypes.c_double * 12)()
    la_arr = (ctypes.c_int64 * 12)()
    L.fmm_profile(plan._h, 1)
    plan.rebuild(X)
    plan.eval(Q, out=(phi, g))
    L.fmm_profile_read(plan._h, ms_arr, la_arr)
    sz = plan.sizes()
    plan.close()
    n = Q.shape[0]
    return {"theta": theta, "value": n / (ms / 1e3), "unit": UNIT, "ms": ms,
            "eval_only": {"value": n / (ms_eval / 1e3), "ms": ms_eval},
            "rel_error_vs_direct": err, "m2l_pairs": sz["nv"], "p2p_leaf_pairs": sz["nu"],
            "pass_ms": {PASSES[i]: ms_arr[i] for i in range(12)},
            "lists_over_dual_speedup": ms / ms_lists,
            "lists_over_dual_speedup_eval_only": ms_eval / ms_eval_lists}


def err_stats(phi, grad, ref_phi, ref_grad, reference):
    """Relative L2 error over the sampled targets and the largest relative
    error of one target, for phi and for grad phi (vector norm per target)."""
    dphi = np.abs(phi - ref_phi)
    dg = np.linalg.norm(grad - ref_grad, axis=1)
    gn = np.linalg.norm(ref_grad, axis=1)
    return {"phi": float(np.linalg.norm(phi - ref_phi) / np.linalg.norm(ref_phi)),
            "grad": float(np.linalg.norm(grad - ref_grad) / np.linalg.norm(ref_grad)),
            "phi_max_target": float(np.max(dphi / np.abs(ref_phi))),
            "grad_max_target": float(np.max(dg / np.where(gn > 0, gn, 1.0))),
            "targets": int(len(ref_phi)), "reference": reference}


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1602_02244_gb300 import binding, build, workloads
    build.build()
    L = binding.library()
    L.fmm_kernel_launches.restype = ctypes.c_uint64
    L.fmm_profile.argtypes = [ctypes.c_void_p, ctypes.c_int]
    L.fmm_profile_read.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_int64)]

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    n, p, S = args.n, args.order, args.leaf
    xyz_np, q_np = workloads.plummer_problem(n, rank)
    w_np = workloads.rng(2).normal(size=n)  # loss weights: L = sum w_i phi_i
    X = torch.tensor(xyz_np, device=dev)
    Q = torch.tensor(q_np, device=dev)
    W = torch.tensor(w_np, device=dev)
    wx = args.wx_direct == "on"
    plan = binding.Plan(X, leaf_size=S, order=p, precision=args.precision,
                        m2l_path=args.m2l_path, p2p_tile=args.p2p_tile,
                        m2l_tile=args.m2l_tile, wx_direct=wx)  # S = 0: autotune
    S = plan.sizes()["leaf_size"]
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    grad = torch.empty(n, 3, dtype=torch.float64, device=dev)
    dq = torch.empty(n, dtype=torch.float64, device=dev)
    dx = torch.empty(n, 3, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        plan.rebuild(X)
        plan.eval(Q, out=(phi, grad))
        plan.adjoint(W, Q, grad_q=grad, out=(dq, dx))

    evals_per_step = 2  # the forward mat-vec and the adjoint's mat-vec with the weights
    for _ in range(max(args.warmup, 3)):
        step()
    pairs, v_pairs, layout = algorithmic_work(plan)
    tiles = plan.tiles()
    m2l_form = tiles["m2l_tile"]
    sizes = plan.sizes()
    fp32_peak = binding.fp32_peak()  # TFLOP/s, measured on this GPU just before the timed steps
    ms_arr = (ctypes.c_double * 12)()
    la_arr = (ctypes.c_int64 * 12)()
    L.fmm_profile(plan._h, 1)
    L.fmm_profile_read(plan._h, ms_arr, la_arr)  # reset
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    l0 = L.fmm_kernel_launches()
    t_wall0 = time.perf_counter()
    step_ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)  # L2 flush (256 MB write), outside the timed events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    barrier()
    t_wall = time.perf_counter() - t_wall0
    launches = int(L.fmm_kernel_launches() - l0)
    clk = clocks.stop()
    L.fmm_profile_read(plan._h, ms_arr, la_arr)
    L.fmm_profile(plan._h, 0)
    pass_ms = {PASSES[i]: ms_arr[i] / args.steps for i in range(12)}
    pass_launch = {PASSES[i]: la_arr[i] / args.steps for i in range(12)}
    ms = max_over_ranks(float(np.mean(step_ms)), world, dev)
    value = n * world / (ms / 1e3)

    # error statement, first against the GPU's FP64 brute-force sum
    # (fmm_direct) on 4096 sampled targets; the CPU-baseline leg below adds
    # the oracle's FP64 direct sum at the same targets
    sel = workloads.sample_targets(n, 4096, 1)
    sel_t = torch.tensor(sel, device=dev)
    pd, gd = binding.direct(X, Q, X[sel_t])
    pd, gd = pd.cpu().numpy(), gd.cpu().numpy()

    def rel_err(ph, gr):
        return err_stats(ph.cpu().numpy()[sel], gr.cpu().numpy()[sel], pd, gd,
                         "fmm_direct (GPU, FP64 brute force)")

    err_mixed = rel_err(phi, grad)
    phi_s, grad_s = phi.cpu().numpy()[sel], grad.cpu().numpy()[sel]

    # roofline of the dominant pass
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    max_mhz = clk.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_nominal = sms * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12  # TFLOP/s
    nc = (p + 1) ** 2
    work = {"P2P": ("alu", evals_per_step * 20.0 * pairs / 1e12, "TFLOP/s", fp32_peak),
            "M2L": ("alu", evals_per_step * 2.0 * nc * nc * v_pairs / 1e12, "TFLOP/s", fp32_peak)}
    m2l_tensor = args.precision == "mixed" and p <= 10 and args.m2l_path != "simt"
    if m2l_tensor:
        # the tensor peak of the operand form: FP16 (kind::f16) runs at the
        # measured sustained bf16 rate, TF32 at that rate x the nominal
        # tf32/bf16 ratio (1.1 / 2.25 dense PFLOP/s); algorithmic flops count
        # one product, not the three of the hi/lo split
        bf16_peak = peaks.get("bf16_tflops_sustained", 1700.0)
        tc_peak = bf16_peak if m2l_form == 2 else bf16_peak * 1.1 / 2.25
        work["M2L"] = ("tensor", evals_per_step * 2.0 * nc * nc * v_pairs / 1e12, "TFLOP/s",
                       tc_peak)
    # bandwidth-bound passes: algorithmic bytes (read + write once) per step
    hbm = peaks.get("hbm_gbs", 6800.0)
    nleaves = int(np.sum(layout["box_nchild"] == 0))
    nb = sizes["nboxes"]
    cb = 4 if args.precision == "mixed" else 8
    e = evals_per_step
    hbm_bytes = {"keys+sort": n * (24 + 12) + 8 * 2 * n * 12,   # keys; 8 radix passes
                 "P2M": e * (n * 16 + nleaves * nc * cb),
                 "M2M": e * 2 * nb * nc * cb,
                 "L2L": e * 2 * nb * nc * cb,
                 "L2P": e * (n * 16 + nleaves * nc * cb + n * 4 * cb),  # far field at cb bytes
                 # the adjoint's dL/dx (w, q, dL/dq-side gradients in, dx out);
                 # in mixed precision the per-target far + near sum is part of P2P
                 "reduce": n * (16 + 24 + 24 + 24) if args.precision == "mixed"
                 else e * (n * 64 + n * 32) + n * (16 + 24 + 24 + 24)}
    for k, bts in hbm_bytes.items():
        work[k] = ("hbm", bts / 1e9, "GB/s", hbm)
    dom = max(pass_ms, key=pass_ms.get)
    if dom in work:
        bound, units, unit, peak = work[dom]
        achieved = units / (pass_ms[dom] / 1e3)
    else:
        bound, unit, peak = "hbm", "GB/s", hbm
        achieved = None
    roof = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": (achieved / peak) if achieved else None,
            "traffic": TRAFFIC_BYTES.get((dom, n, p, S, args.precision, tiles["p2p_tile"], wx))
                       if dom == "P2P" else None,
            "peak_source": ("FP32: fmm_fp32_peak, paired-FMA chains on this GPU (of measured); "
                            "nominal %d SMs x %d lanes x 2 flop x %.0f MHz = %.1f TFLOP/s"
                            % (sms, FP32_LANES_PER_SM, max_mhz, fp32_nominal)
                            if bound == "alu" else
                            ("FP16 = measured sustained bf16 (of measured)" if m2l_form == 2 else
                             "TF32 = measured sustained bf16 x 1.1/2.25 (of measured)")
                            if bound == "tensor"
                            else "MEASURED_PEAKS.json hbm_gbs (of measured)")}
    if bound == "alu" and achieved:
        roof["frac_of_nominal"] = achieved / fp32_nominal
    other = {k: {"bound": v[0], "achieved": v[1] / (pass_ms[k] / 1e3), "unit": v[2],
                 "peak": v[3], "frac": v[1] / (pass_ms[k] / 1e3) / v[3]}
             for k, v in work.items() if pass_ms.get(k)}
    if pass_ms.get("M2L"):
        # M2L bytes: the gathered source multipoles read once and the locals
        # written once per evaluation, plus the operator table
        m2l_bytes = e * (2 * nb * nc * cb) + 343 * nc * nc * cb
        other["M2L_hbm"] = {"bound": "hbm", "achieved": m2l_bytes / 1e9 / (pass_ms["M2L"] / 1e3),
                            "unit": "GB/s", "peak": hbm,
                            "frac": m2l_bytes / 1e9 / (pass_ms["M2L"] / 1e3) / hbm}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": "Plummer N=%d, charges 1/N, p=%d, leaf %d (%s), %s precision; "
                                   "step = plan (keys, sort, octree, U/V/W/X lists) + forward "
                                   "(phi and grad) + adjoint of L = sum w phi (dL/dq, dL/dx; "
                                   "forward gradient stored)"
                                   % (n, p, S, "autotuned" if args.leaf == 0 else "fixed",
                                      args.precision),
                       "m2l": ("tensor cores (tcgen05 kind::tf32, three-product TF32 split)"
                               if args.m2l_tile == 1 else
                               "tensor cores (tcgen05 kind::f16, three-product FP16 split with "
                               "power-of-two scalings)")
                              if m2l_tensor
                              else "CUDA cores",
                       "wx_direct": ("W/X pairs of two leaves whose W leaf holds <= (p+1)^2 "
                                     "points by the direct sum" if wx else "off"),
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "256 MB flush between steps; working set >> L2",
                       "boxes": sizes["nboxes"], "levels": sizes["nlevels"], "U": sizes["nu"],
                       "V": sizes["nv"], "W": sizes["nw"], "X": sizes["nx"],
                       "p2p_pairs": pairs, "tiles": tiles},
            "clocks": clk, "gpu_launches": launches, "wall_s_timed": t_wall,
            "pass_ms": pass_ms, "pass_launches": pass_launch, "roofline": roof,
            "pass_roofline": other, "fp32_peak_tflops": fp32_peak,
            "rel_error_vs_direct": err_mixed}

    # plan + forward only, and the mat-vecs without the plan (the paper's
    # mat-vec application time)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.rebuild(X)
        plan.eval(Q, out=(phi, grad))
    e1.record(stream)
    e1.synchronize()
    ms_pf = e0.elapsed_time(e1) / args.steps
    line["plan_forward"] = {"value": n / (ms_pf / 1e3), "unit": UNIT, "ms": ms_pf}
    e0.record(stream)
    for _ in range(args.steps):
        plan.eval(Q, out=(phi, grad))
    e1.record(stream)
    e1.synchronize()
    ms_eval = e0.elapsed_time(e1) / args.steps
    line["eval_only"] = {"value": n / (ms_eval / 1e3), "unit": UNIT, "ms": ms_eval}
    e0.record(stream)
    for _ in range(args.steps):
        plan.eval(Q, out=(phi, grad))
        plan.adjoint(W, Q, grad_q=grad, out=(dq, dx))
    e1.record(stream)
    e1.synchronize()
    ms_fa = e0.elapsed_time(e1) / args.steps
    line["fwd_adjoint"] = {"value": n / (ms_fa / 1e3), "unit": UNIT, "ms": ms_fa}

    # end to end through the C-ABI on pinned host buffers
    if not args.no_e2e:
        hx = torch.tensor(xyz_np).pin_memory()
        hq = torch.tensor(q_np).pin_memory()
        hw = torch.tensor(w_np).pin_memory()
        hphi = torch.empty(n, dtype=torch.float64).pin_memory()
        hg = torch.empty(n, 3, dtype=torch.float64).pin_memory()
        hdq = torch.empty(n, dtype=torch.float64).pin_memory()
        hdx = torch.empty(n, 3, dtype=torch.float64).pin_memory()

        def host_step():
            plan.solve_adjoint_host_ptr(hx.data_ptr(), hq.data_ptr(), hw.data_ptr(), n,
                                        hphi.data_ptr(), hg.data_ptr(), hdq.data_ptr(),
                                        hdx.data_ptr())

        for _ in range(2):
            host_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_step()
        t_e2e = max_over_ranks((time.perf_counter() - t0) / args.steps, world, dev)
        line["e2e"] = {"value": n * world / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 40 * n,
                       "d2h_bytes_per_step": 64 * n, "ms": 1e3 * t_e2e}

    # plain FP64 GPU FMM at the smallest order whose direct-sum error is no
    # larger than the mixed-precision result's, the same step timed
    if not args.no_fp64 and args.precision == "mixed":
        phi64 = torch.empty_like(phi)
        g64 = torch.empty_like(grad)
        dq64 = torch.empty_like(dq)
        dx64 = torch.empty_like(dx)
        tried = []
        for p64 in range(max(2, p - 3), 13):
            plan64 = binding.Plan(X, leaf_size=S, order=p64, precision="fp64", wx_direct=wx)
            plan64.eval(Q, out=(phi64, g64))
            e64 = rel_err(phi64, g64)
            tried.append({"order": p64, "phi": e64["phi"]})
            if e64["phi"] <= err_mixed["phi"] or p64 == 12:
                break
            plan64.close()
        plan64.adjoint(W, Q, grad_q=g64, out=(dq64, dx64))
        barrier()
        reps = 2
        e0.record(stream)
        for _ in range(reps):
            plan64.rebuild(X)
            plan64.eval(Q, out=(phi64, g64))
            plan64.adjoint(W, Q, grad_q=g64, out=(dq64, dx64))
        e1.record(stream)
        e1.synchronize()
        ms64 = e0.elapsed_time(e1) / reps
        e0.record(stream)
        plan64.eval(Q, out=(phi64, g64))
        e1.record(stream)
        e1.synchronize()
        ms64_eval = e0.elapsed_time(e1)
        line["fp64_equal_error"] = {"order": p64, "value": n / (ms64 / 1e3), "unit": UNIT,
                                    "ms": ms64, "eval_only_ms": ms64_eval,
                                    "rel_error_vs_direct": e64, "orders_tried": tried,
                                    "mixed_speedup": ms64 / ms,
                                    "mixed_speedup_eval_only": ms64_eval / ms_eval}
        line["config"]["fp64_equal_error"] = {"order": p64, "ms_per_step": ms64,
                                              "mixed_speedup": ms64 / ms}
        plan64.close()

    if args.dual_theta > 0:
        line["dual_tree"] = dual_leg(X, Q, S, p, args.precision, args.dual_theta, rel_err,
                                     min(args.steps, 5), stream, ms_pf, ms_eval)
    if not args.no_batch:
        line["batched"] = batched_leg(dev, args.steps, args.warmup, args.batch_leaf, wx)
    if not args.no_lattice:
        line["lattice"] = lattice_leg(dev)
    if args.precond:
        line["precond"] = precond_leg(dev)
        line["precond_helmholtz"] = helmholtz_precond_rows(dev)
    if not args.no_helmholtz and rank == 0 and world == 1:
        line["helmholtz"] = helmholtz_leg(dev, L)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ncpu = args.cpu_sample or n
        cpu, ref = cpu_baseline(ncpu, p, S, sel if ncpu == n else workloads.sample_targets(ncpu, 4096, 1),
                                direct_wx=(p + 1) ** 2 if wx else 0)
        line["cpu_baseline"] = cpu
        if ncpu == n:
            # the error statement against the oracle: its FP64 direct sum at
            # the same 4096 sampled targets
            line["rel_error_vs_oracle_direct"] = err_stats(phi_s, grad_s, ref[0], ref[1],
                                                           "oracle direct sum (CPU, FP64)")
            line["fmm_direct_vs_oracle_direct"] = err_stats(pd, gd, ref[0], ref[1],
                                                            "oracle direct sum (CPU, FP64)")
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
