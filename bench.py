"""Benchmark: TT-sGMRES time-to-residual 1e-6 on one GB300.

Workload (the convection-diffusion system the metric is quoted on): d = 10
modes of n = 64, ``A = sum_k I x .. x (L + 10 B) x .. x I`` with
``L = (n+1)^2 tridiag(-1, 2, -1)`` and ``B = (n+1)/2 tridiag(-1, 0, 1)`` (TT
operator rank 2), b a random TT of rank 4 (seeded Gaussian cores), basis rank
cap 64, Krylov cap 80 per cycle, s = 160 Khatri-Rao sketch rows, oversampling
10, true relative residual target 1e-6.

One "step" is one whole solve (all hot-path rows: matvec, sketch, inner
products, randomized rounding with FP64 QR, sketched least squares, restarts
and the FP64 residual check) with the operator and b resident in HBM.  The
reported ``value`` is seconds per solve (lower is better), timed with CUDA
events on the solver's stream; L2 is flushed (a 512 MiB write) before each step,
outside the timed interval.  ``e2e`` repeats the solve through the public API
with host (pinned) inputs copied in and the solution copied out inside the
timed interval.  With ``--gpus N`` (torchrun) every rank solves its own copy:
the path has no data-parallel split (replicas only).

``--impl reference`` times the FP64 CPU oracle (the same algorithm in NumPy)
on this machine's host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ttinputs as ti  # noqa: E402

METRIC = "TT-sGMRES time-to-residual 1e-6 (s) mixed vs FP64 GPU; contraction TFLOP/s vs peak"
WORKLOAD = "convdiff d=10 n=64 (L+10B Kronecker sum, TT rank 2), b rank 4, rmax 64, m<=80, s=160"
# FP64 and FP32 CUDA-core peaks from the unit counts: 152 SMs x (2 FP64 | 128 FP32)
# FMA/clk x 2 FLOP x 2.070 GHz (maximum SM clock).
FP64_ALU_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# TF32 dense tensor peak = measured BF16 peak x nominal TF32/BF16 ratio (1.1 / 2.25)
TF32_OVER_BF16 = 1.1 / 2.25
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# dominant kernel at this workload, from one ncu capture of the current kernel
# (None once the kernel changes and until it is captured again)
TRAFFIC_BYTES = {"qr_f64": 1.835008e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["tf32", "fp32", "fp64"], default=None)
    ap.add_argument("--no-fp64-leg", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0,
                    help="budget of the host oracle sample")
    ap.add_argument("--case", choices=["solve", "round", "batched"], default="solve",
                    help="'round': time one randomized rounding of w - h v at the workload's "
                         "sizes (the kernel-level case used for ncu captures); 'batched': the "
                         "64-right-hand-side workload through the batched solver")
    ap.add_argument("--workers", type=int, default=16,
                    help="library worker threads (streams) of the batched case")
    ap.add_argument("--seq-sample", type=int, default=4,
                    help="right-hand sides timed one at a time for the batched case's baseline")
    return ap.parse_args()


def workload():
    w = ti.workload("convdiff")
    return w, dict(w.params)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            pk = json.load(f)
        return pk, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def max_over_ranks(value: float, device="cpu") -> float:
    """The slowest rank's timed interval (replicas: every rank solves its own
    copy, so the job takes as long as the slowest one).  Returns ``value``
    unchanged without an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- oracle
def oracle_sample(budget_s: float, mode_note: str):
    """Times the FP64 oracle's TT-sGMRES on the workload for as many Krylov
    iterations as fit in ``budget_s`` (first cycle), and returns seconds per
    iteration plus a description."""
    from oracle import solvers as osol, philox as oph, tt as ott  # noqa: F401
    import oracle.rounding as ornd
    w, p = workload()
    S = oph.sketch_factors(w.ns, p["s"], 0)
    L = p["rmax"] + p["oversample"]
    drm = oph.drm_cores(w.ns, [1] + [L] * (w.d - 1) + [1], 0)
    # run iterations one at a time until the budget is spent
    t0 = time.perf_counter()
    beta = ott.norm(w.b)
    v = ott.scale(w.b, 1.0 / beta)
    Sr0 = ott.sketch_kr_fast(w.b, S)
    Wc = []
    its = 0
    while True:
        wv = ott.matvec(w.op, v)
        Wc.append(ott.sketch_kr_fast(wv, S))
        h = ott.dot(wv, v)
        vt = ornd.rto_round([(1.0, wv), (-h, v)], drm, eps=p["eta"] * 1e-5, rmax=p["rmax"],
                            oversample=p["oversample"])
        v = ott.scale(vt, 1.0 / ott.norm(vt))
        osol.sketched_lstsq(np.stack(Wc, axis=1), Sr0)
        its += 1
        if time.perf_counter() - t0 > budget_s or its >= p["maxit"]:
            break
    dt = time.perf_counter() - t0
    cores = os.cpu_count()
    return dt / its, its, cores, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_iter = []
    its_total = 0
    t_total = 0.0
    budget = max(5.0, args.cpu_seconds / max(1, args.steps))
    for _ in range(args.steps):
        s, its, cores, dt = oracle_sample(budget, "reference")
        per_iter.append(s)
        its_total += its
        t_total += dt
    sec_per_iter = statistics.median(per_iter)
    # a whole solve takes the iteration count the GPU path needs (the same
    # algorithm); the oracle's own count for this workload is of that order
    iters = int(os.environ.get("TTSG_REF_ITERS", "60"))
    value = sec_per_iter * iters
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "host run"},
            "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                             "sample": f"{its_total} Krylov iterations over {args.steps} steps "
                                       f"({t_total:.1f} s), projected to {iters} iterations"},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def run_ours(args):
    import torch
    import torch.distributed as dist
    import paper_2409_09471_gb300 as g
    from paper_2409_09471_gb300._abi import lib
    import ctypes

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    # host oracle sample first (rank 0, single GPU), before any GPU work
    cpu = None
    if rank == 0 and world == 1:
        s_it, its, cores, dt = oracle_sample(args.cpu_seconds, "baseline")
        cpu = (s_it, its, cores, dt)

    mode_name = args.mode or os.environ.get("TTSG_MODE", "tf32")
    mode = {"tf32": g.MODE_TF32, "fp32": g.MODE_FP32, "fp64": g.MODE_FP64}[mode_name]
    w, p = workload()
    op = g.op_to_device(w.op)
    b = g.TT.from_numpy(w.b)
    kw = dict(maxit=p["maxit"], tol=p["tol"], rmax=p["rmax"], s=p["s"], eta=p["eta"],
              stop_safety=0.1, r_sol=p["r_sol"], oversample=p["oversample"], seed=0,
              max_restarts=8)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    # warm-up (the last one profiles every kernel class to find the dominant one)
    ws = None
    info = None
    for i in range(args.warmup):
        if i == args.warmup - 1:
            lib.tt_profile(0xFF)
        x, info = g.tt_sgmres_solve(op, b, mode=mode, workspace=ws, **kw)
        if ws is None:
            ws = torch.empty(info["workspace_bytes"], dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    classes = {0: "gemm", 1: "qr_f64", 2: "jacobi_svd", 3: "lstsq", 4: "misc", 5: "gram_f64",
               6: "chol_f64", 7: "tc_matvec"}
    prof = {}
    for cl in classes:
        ms, nl, fl, by = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        lib.tt_profile_read(cl, ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(fl), ctypes.byref(by))
        prof[classes[cl]] = dict(ms=ms.value, launches=nl.value, flops=fl.value, bytes=by.value)
    dom = max(prof, key=lambda k: prof[k]["ms"])
    dom_cls = [k for k, v in classes.items() if v == dom][0]

    # timed region: the dominant class is event-timed live
    lib.tt_profile(1 << dom_cls)
    clocks = Clocks(local)
    times = []
    iters = []
    launches0 = lib.tt_launch_count()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, info = g.tt_sgmres_solve(op, b, mode=mode, workspace=ws, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        iters.append(info["iters"])
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = lib.tt_launch_count() - launches0
    total_ms = max_over_ranks(sum(times), "cuda")
    ms, nl, fl, by = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    lib.tt_profile_read(dom_cls, ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(fl), ctypes.byref(by))
    lib.tt_profile(0)
    ms_per_step = total_ms / args.steps
    value = ms_per_step / 1e3

    pk, pk_kind = peaks()
    avg_ms = ms.value / max(nl.value, 1)
    fl_per = fl.value / max(nl.value, 1)
    by_per = by.value / max(nl.value, 1)
    if dom == "qr_f64":
        roof = {"bound": "alu", "achieved": fl_per / (avg_ms * 1e-3) / 1e12,
                "peak": FP64_ALU_TFLOPS, "unit": "TFLOP/s",
                "peak_kind": "FP64 CUDA-core peak from unit counts (152 SMs x 2 DFMA/clk x 2.07 GHz)"}
    elif dom == "gemm":
        if mode == g.MODE_TF32:
            peak_c = pk["bf16_tflops_sustained"] * TF32_OVER_BF16
            kind = f"{pk_kind} BF16 sustained x 1.1/2.25 (TF32)"
            bound = "tensor"
        elif mode == g.MODE_FP32:
            peak_c, kind, bound = FP32_ALU_TFLOPS, "FP32 CUDA-core peak from unit counts", "alu"
        else:
            peak_c, kind, bound = FP64_ALU_TFLOPS, "FP64 CUDA-core peak from unit counts", "alu"
        ai = fl_per / max(by_per, 1)
        if ai < peak_c * 1e12 / (pk["hbm_gbs"] * 1e9):
            roof = {"bound": "hbm", "achieved": by_per / (avg_ms * 1e-3) / 1e9,
                    "peak": pk["hbm_gbs"], "unit": "GB/s", "peak_kind": f"{pk_kind} copy bandwidth"}
        else:
            roof = {"bound": bound, "achieved": fl_per / (avg_ms * 1e-3) / 1e12, "peak": peak_c,
                    "unit": "TFLOP/s", "peak_kind": kind}
    else:
        roof = {"bound": "hbm", "achieved": by_per / (avg_ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "peak_kind": f"{pk_kind} copy bandwidth"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = TRAFFIC_BYTES.get(dom)
    roof["kernel"] = dom
    roof["launches_per_step"] = nl.value / args.steps
    roof["avg_launch_us"] = avg_ms * 1e3
    roof["share_of_step"] = ms.value / total_ms if total_ms > 0 else None

    # FP64 GPU leg (the "mixed vs FP64 GPU" comparison): one solve
    fp64 = None
    if not args.no_fp64_leg and mode != g.MODE_FP64:
        xf, inf64 = g.tt_sgmres_solve(op, b, mode=g.MODE_FP64, **kw)
        torch.cuda.synchronize()
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xf, inf64 = g.tt_sgmres_solve(op, b, mode=g.MODE_FP64, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64 = dict(seconds=e0.elapsed_time(e1) / 1e3, iters=inf64["iters"],
                    true_res=inf64["true_res"], cycles=inf64["cycles"])

    # end to end: pinned host inputs in, solution out, inside the timed interval
    op_h = [c.cpu().pin_memory() for c in op]
    b_h = [c.cpu().pin_memory() for c in b.cores]
    op_d = [torch.empty_like(c) for c in op]
    b_d = [torch.empty_like(c) for c in b.cores]
    h2d = sum(c.numel() * c.element_size() for c in op_h + b_h)
    e2e_ms, d2h = [], 0
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for hsrc, ddst in zip(op_h + b_h, op_d + b_d):
            ddst.copy_(hsrc, non_blocking=True)
        xe, ie = g.tt_sgmres_solve(op_d, g.TT(b_d), mode=mode, workspace=ws, **kw)
        outs = [c.to("cpu", non_blocking=True) for c in xe.cores]
        res_h = torch.tensor([ie["true_res"]])
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
        d2h = sum(o.numel() * o.element_size() for o in outs)

    # the contraction half of the metric: algorithmic TFLOP/s of the tcgen05
    # matvec (against the TF32 tensor peak; the split-TF32 scheme issues three
    # products per algorithmic one) and of the CUDA-core GEMMs (against the FP32
    # unit peak), from the profiled warm-up step
    contraction = {}
    for key, peak_c, kind in (("tc_matvec", pk["bf16_tflops_sustained"] * TF32_OVER_BF16,
                               f"{pk_kind} BF16 sustained x 1.1/2.25 (TF32 tensor)"),
                              ("gemm", FP32_ALU_TFLOPS, "FP32 CUDA-core peak from unit counts")):
        v = prof[key]
        if v["ms"] > 0 and v["launches"] > 0:
            tf = v["flops"] / (v["ms"] * 1e-3) / 1e12
            contraction[key] = {"tflops": tf, "peak": peak_c, "frac": tf / peak_c,
                                "peak_kind": kind, "launches": v["launches"],
                                "avg_launch_us": v["ms"] * 1e3 / v["launches"]}
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"tf32": "tf32+f64", "fp32": "f32+f64", "fp64": "f64"}[mode_name],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "mode": mode_name, "parallelism": "replicas",
                       "l2": "flushed (512 MiB write) before every step"},
            "iters_per_solve": statistics.median(iters), "true_res": info["true_res"],
            "svd_nonconverged": info.get("svd_nonconverged"),
            "svd_sweeps": {"max": info.get("svd_max_sweeps"),
                           "mean": round(info.get("svd_mean_sweeps") or 0.0, 2)},
            "cycles": info["cycles"], "max_rank": info["max_rank"],
            "gpu_launches": int(launches), "roofline": roof, "contraction": contraction,
            "kernel_time_ms_by_class_warmup": {k: round(v["ms"], 3) for k, v in prof.items()},
            "e2e": {"value": statistics.mean(e2e_ms) / 1e3, "unit": "s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "clocks": clk}
    if fp64:
        line["fp64_gpu"] = fp64
        line["speedup_vs_fp64_gpu"] = fp64["seconds"] / value
    if cpu is not None:
        s_it, its, cores, dt = cpu
        proj = s_it * statistics.median(iters)
        line["cpu_baseline"] = {"value": proj, "unit": "s", "cores": cores, "kind": "oracle",
                                "sample": f"{its} Krylov iterations of the FP64 oracle's first "
                                          f"cycle ({dt:.1f} s), projected to the GPU solve's "
                                          f"{statistics.median(iters)} iterations"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_round_case(args):
    """One Gram-Schmidt rounding of the solver at the workload's sizes:
    ``Round(A v - h v)`` with v a random rank-64 TT (d=10, n=64), rank cap 64,
    oversampling 10, tolerance 1e-7, in the selected mode."""
    import torch
    import paper_2409_09471_gb300 as g
    mode_name = args.mode or "fp32"
    mode = {"tf32": g.MODE_TF32, "fp32": g.MODE_FP32, "fp64": g.MODE_FP64}[mode_name]
    w, p = workload()
    dt = g.mode_dtype(mode)
    v = g.TT.from_numpy(ti.random_tt(w.ns, [1] + [64] * (w.d - 1) + [1], seed=5), dt)
    Av = g.tt_matvec(g.op_to_device(w.op, dt), v, mode=mode)
    times = []
    for i in range(args.warmup + args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        y = g.tt_round_rand([Av, v], [1.0, -0.3], 1e-7, 64, 10, seed=1, mode=mode)
        e1.record()
        torch.cuda.synchronize()
        if i >= args.warmup:
            times.append(e0.elapsed_time(e1))
    print(json.dumps({"case": "round", "mode": mode_name, "ms_per_call": statistics.median(times),
                      "out_ranks": y.ranks}), flush=True)


def run_batched_case(args):
    """The batched workload: 64 right-hand sides (d=8, n=32 Laplacian, bond
    ranks U{1..12}, rank cap 150), solved by the library's worker pool in the
    selected mode; one JSON line with the whole-batch time and RHS/s."""
    import torch
    import paper_2409_09471_gb300 as g
    mode_name = args.mode or "tf32"
    mode = {"tf32": g.MODE_TF32, "fp32": g.MODE_FP32, "fp64": g.MODE_FP64}[mode_name]
    w = ti.workload("batched")
    p = w.params
    op = g.op_to_device(w.op)
    bs = [g.TT.from_numpy(b) for b in w.b]
    kw = dict(maxit=p["maxit"], tol=p["tol"], rmax=p["rmax"], mode=mode, s=p["s"],
              round_tol=p["round_tol"], r_sol=p["r_sol"], oversample=p["oversample"],
              max_restarts=10, nworkers=args.workers)
    times = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = g.tt_sgmres_solve_batched(op, bs, **kw)
        torch.cuda.synchronize()
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    st = [r[1]["status"] for r in res]
    tr = [r[1]["true_res"] for r in res]
    it = [r[1]["iters"] for r in res]
    sec = statistics.median(times)
    # the same right-hand sides one at a time through the single-RHS solver
    # (a bounded sample, projected to the batch by the batch's iteration counts)
    seq_kw = {k: v for k, v in kw.items() if k != "nworkers"}
    seq_t, seq_it = 0.0, 0
    for b in bs[:args.seq_sample]:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, inf = g.tt_sgmres_solve(op, b, **seq_kw)
        torch.cuda.synchronize()
        seq_t += time.perf_counter() - t0
        seq_it += inf["iters"]
    line = {"case": "batched", "mode": mode_name, "nrhs": len(bs), "workers": args.workers,
            "seconds": sec, "rhs_per_s": len(bs) / sec,
            "not_converged": int(sum(s != 0 for s in st)), "max_true_res": max(tr),
            "iters_mean": float(np.mean(it)), "iters_max": int(max(it))}
    if seq_it:
        proj = seq_t / seq_it * float(np.sum(it))
        line["sequential"] = {"sample_rhs": args.seq_sample, "sample_seconds": seq_t,
                              "projected_seconds": proj, "batched_speedup": proj / sec}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.case == "round":
        run_round_case(args)
        return
    if args.case == "batched":
        run_batched_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
