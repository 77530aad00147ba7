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
on this machine's host cores: one full solve of the same workload (restarts,
final rounding and exact residual included), reported as K equal steps; the
warm-up steps are single untimed Krylov iterations.  The GPU arm's
``cpu_baseline`` is one such full solve.  ``roofline`` comes from a separate pass of solves in
which every kernel launch is bracketed by CUDA events; the headline loop runs
without them.
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
    ap.add_argument("--mode", choices=["tf32", "bf16", "fp32", "fp64"], default=None)
    ap.add_argument("--no-fp64-leg", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the host oracle solve of the GPU arm")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other configurations' solves")
    ap.add_argument("--ref-small", action="store_true",
                    help="reference arm on a d=4, n=12 system (plumbing tests only)")
    ap.add_argument("--case", choices=["solve", "round", "batched"], default="solve",
                    help="'round': time one randomized rounding of w - h v at the workload's "
                         "sizes (the kernel-level case used for ncu captures); 'batched': the "
                         "64-right-hand-side workload through the batched solver")
    ap.add_argument("--round-workload", choices=["convdiff", "large_rank"], default="convdiff",
                    help="sizes of the 'round' case: the bench workload (d=10, n=64, rank 64) or "
                         "the large-rank one (d=20, n=128, rank 128)")
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
def oracle_params(p):
    """Solver settings of the FP64 oracle run that match the GPU solve: the
    rounding tolerance of the first cycle (eta * stop_safety * tol) and the
    DRM capacity the GPU draws (largest rank cap plus oversampling)."""
    return dict(maxit=p["maxit"], tol=p["tol"], round_tol=p["eta"] * 0.1 * p["tol"],
                rmax=p["rmax"], oversample=p["oversample"], r_sol=p["r_sol"], stop_safety=0.1,
                max_restarts=8)


def oracle_inputs(w, p):
    from oracle import philox as oph
    S = oph.sketch_factors(w.ns, p["s"], 0)
    rb = max(max(c.shape[0], c.shape[2]) for c in w.b)
    L = max(p["rmax"], p["r_sol"], rb) + p["oversample"]
    drm = oph.drm_cores(w.ns, [1] + [L] * (w.d - 1) + [1], 0)
    return S, drm


def oracle_full_solve(w, p):
    """One full FP64 oracle TT-sGMRES solve of the workload on the host cores:
    every Krylov iteration, restarts, the final rounding and the exact FP64
    residual check, timed as a whole.  Returns (seconds, info)."""
    from oracle import solvers as osol
    S, drm = oracle_inputs(w, p)
    t0 = time.perf_counter()
    _, info = osol.solve(w.op, w.b, S, drm, **oracle_params(p))
    return time.perf_counter() - t0, info


def oracle_warmup(w, p):
    """One untimed Krylov iteration of the oracle (warms the BLAS threads)."""
    from oracle import solvers as osol
    S, drm = oracle_inputs(w, p)
    q = oracle_params(p)
    osol.tt_sgmres(w.op, w.b, S, drm, maxit=1, tol=q["tol"], round_tol=q["round_tol"],
                   rmax=q["rmax"], oversample=q["oversample"], r_sol=q["r_sol"])


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def ref_workload(args):
    """The bench workload, or (``--ref-small``, a plumbing-test option) the
    same system at d = 4, n = 12."""
    if args.ref_small:
        w = ti.workload("convdiff", d=4, n=12, maxit=30)
        return w, dict(w.params), "convdiff d=4 n=12 (plumbing test)"
    w, p = workload()
    return w, p, WORKLOAD


def run_reference(args):
    """The reference arm: the FP64 oracle (the same algorithm in NumPy), as it
    stands, on the host cores.  The timed region is one full solve (every
    Krylov iteration, restarts, the final rounding and the exact residual),
    about 40 s on 16 Grace cores; its K steps are the K equal shares of that
    solve, so that ``ms_per_step * steps`` is the timed duration and the run
    ends within a minute for any K.  ``value`` is the solve's time, the
    metric's seconds per solve."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w, p, name = ref_workload(args)
    for _ in range(args.warmup):
        oracle_warmup(w, p)
    value, info = oracle_full_solve(w, p)
    cores = host_cores()
    steps = max(1, args.steps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s",
            "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
            "ms_per_step": value * 1e3 / steps, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name, "l2": "host run",
                       "step": f"1/{steps} of one timed full solve"},
            "iters_per_solve": info["iters"], "true_res": info["true_res"],
            "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                             "sample": "1 full FP64 oracle solve (every iteration, restarts, "
                                       "final rounding, exact residual), timed as a whole; "
                                       f"warm-up: {args.warmup} single untimed Krylov "
                                       "iterations"},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def measured_alu_peaks(torch):
    """FP64 and FP32 (no TF32) GEMM rates of cuBLAS on this GPU, best of three
    back-to-back calls each, in TFLOP/s: the CUDA-core peaks the FP64 QR and the
    FP32 CUDA-core GEMMs are held against."""
    out = {}
    old = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt, n in (("fp64", torch.float64, 4096), ("fp32", torch.float32, 8192)):
            a = torch.randn(n, n, dtype=dt, device="cuda")
            b = torch.randn(n, n, dtype=dt, device="cuda")
            torch.matmul(a, b)
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) * 1e-3)
            out[name] = 2.0 * n ** 3 / best / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    return out


CLASSES = {0: "gemm", 1: "qr_f64", 2: "jacobi_svd", 3: "lstsq", 4: "misc", 5: "gram_f64",
           6: "chol_f64", 7: "tc_matvec"}


def read_profile(lib, ctypes):
    prof = {}
    for cl, name in CLASSES.items():
        ms, nl, fl, by = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        lib.tt_profile_read(cl, ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(fl), ctypes.byref(by))
        prof[name] = dict(ms=ms.value, launches=nl.value, flops=fl.value, bytes=by.value)
    return prof


def timed_solves(torch, g, op, b, kw, ws, steps, flush, stream):
    times, infos = [], []
    for _ in range(steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, info = g.tt_sgmres_solve(op, b, workspace=ws, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
        infos.append(info)
    return times, infos, x


def extra_configs(torch, g, flush, stream, modes):
    """The other configurations' solves (not part of the headline): the FP64
    Laplacian (d = 4, n = 16), the headline system in split-BF16 mode, the
    large-rank Laplacian (d = 20, n = 128, rank
    cap 128) in the mixed mode and in FP64, the preconditioned Markov-chain
    system (d = 5, n = 128) in FP64 and FP32, the 64-right-hand-side batch
    (d = 8, n = 32) through the worker pool, and one forward + adjoint solve
    of the differentiable workload (d = 12, n = 64)."""
    out = {}

    def solve_cfg(name, mode, reps):
        w = ti.workload(name)
        p = w.params
        op = g.op_to_device(w.op)
        b = g.TT.from_numpy(w.b)
        kw = dict(maxit=p["maxit"], tol=p["tol"], rmax=p["rmax"], mode=mode, s=p["s"],
                  round_tol=p.get("round_tol", 0.0), eta=p.get("eta", 0.1),
                  stop_safety=0.01 if name == "laplace_fp64" else 0.1, r_sol=p["r_sol"],
                  oversample=p["oversample"], seed=0, max_restarts=8)
        x, info = g.tt_sgmres_solve(op, b, **kw)  # warm (allocates the workspace)
        ws = torch.empty(info["workspace_bytes"], dtype=torch.uint8, device="cuda")
        t, infos, _ = timed_solves(torch, g, op, b, kw, ws, reps, flush, stream)
        del ws
        torch.cuda.empty_cache()
        inf = infos[-1]
        return {"seconds": statistics.median(t), "iters": inf["iters"], "cycles": inf["cycles"],
                "true_res": inf["true_res"], "max_rank": inf["max_rank"], "runs": reps}

    out["laplace_fp64_d4_n16"] = {"fp64": solve_cfg("laplace_fp64", g.MODE_FP64, 3)}
    # the headline workload with the split-BF16 tensor-core matvec
    out["convdiff_d10_n64_bf16"] = {"bf16": solve_cfg("convdiff", g.MODE_BF16, 3)}
    lr = {}
    for mname in modes:
        lr[mname] = solve_cfg("large_rank", {"tf32": g.MODE_TF32, "fp32": g.MODE_FP32,
                                             "fp64": g.MODE_FP64}[mname], 2)
    if "fp64" in lr:
        for mname in lr:
            if mname != "fp64":
                lr[mname]["speedup_vs_fp64_gpu"] = lr["fp64"]["seconds"] / lr[mname]["seconds"]
    out["large_rank_d20_n128"] = lr
    # Markov chain (d = 5 coupled random walks of n = 128 states, the paper's
    # smallest size, at its rank cap 80), right-preconditioned by the
    # exponential sum of the shifted independent part; the shift is a third of
    # the smallest spectral gap in FP64 and the whole gap in FP32 (the float
    # products cannot resolve the 1/sigma amplification of a smaller shift)
    w = ti.workload("markov", n=128)
    p = w.params
    op = g.op_to_device(w.op)
    b = g.TT.from_numpy(w.b)
    mk = {}
    for mname, mval, frac in (("fp64", g.MODE_FP64, 0.3), ("fp32", g.MODE_FP32, 1.0)):
        blocks, a, bnd = ti.markov_precond_blocks(w.extra["Q"], shift_frac=frac)
        P = g.Precond.for_interval(a, bnd, 1e-2, [torch.as_tensor(B, device="cuda") for B in blocks])
        kw = dict(maxit=p["maxit"], tol=p["tol"], rmax=80, mode=mval, s=p["s"], eta=p["eta"],
                  r_sol=80, oversample=p["oversample"], seed=0, max_restarts=20)
        g.tt_spgmres_solve(op, P, b, **kw)  # warm
        ts = []
        for _ in range(2):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, inf = g.tt_spgmres_solve(op, P, b, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        mk[mname] = {"seconds": statistics.median(ts), "iters": inf["iters"],
                     "cycles": inf["cycles"], "true_res": inf["true_res"],
                     "max_rank": inf["max_rank"], "precond_terms": len(P.alpha),
                     "shift_of_gap": frac}
    out["markov_d5_n128_preconditioned_rank80"] = mk
    # the batched workload: all 64 right-hand sides (d = 8, n = 32 Laplacian,
    # bond ranks U{1..12}, rank cap 150) through the library's worker pool,
    # FP32 contractions (with the split-TF32 matvec the hardest right-hand
    # side levels off near the 1e-6 target at this rank cap), one timed batch
    # after a warm call on two right-hand sides
    w = ti.workload("batched")
    p = w.params
    op = g.op_to_device(w.op)
    bs = [g.TT.from_numpy(b) for b in w.b]
    kw = dict(maxit=p["maxit"], tol=p["tol"], rmax=p["rmax"], mode=g.MODE_FP32, s=p["s"],
              round_tol=p["round_tol"], r_sol=p["r_sol"], oversample=p["oversample"],
              max_restarts=20, nworkers=16)
    g.tt_sgmres_solve_batched(op, bs[:2], **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = g.tt_sgmres_solve_batched(op, bs, **kw)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    out["batched_d8_n32_64rhs"] = {"fp32": {
        "seconds": sec, "rhs_per_s": len(bs) / sec, "workers": 16,
        "not_converged": int(sum(i["status"] != 0 for _, i in res)),
        "max_true_res": max(i["true_res"] for _, i in res),
        "iters_mean": float(np.mean([i["iters"] for _, i in res])),
        "iters_max": int(max(i["iters"] for _, i in res))}}
    del res, bs, op
    torch.cuda.empty_cache()
    # differentiable workload: forward solve + adjoint solve + backward contractions
    w = ti.workload("differentiable")
    p = w.params
    theta = torch.tensor(w.extra["theta"], dtype=torch.float64, device="cuda", requires_grad=True)
    M = torch.as_tensor(w.extra["L"], device="cuda")
    bc = [torch.as_tensor(c, device="cuda").requires_grad_(True) for c in w.b]
    xt = [torch.as_tensor(c, device="cuda") for c in w.extra["x_target"]]
    kw = dict(maxit=p["maxit"], tol=1e-8, rmax=p["rmax"], mode=g.MODE_FP32, r_sol=p["r_sol"],
              oversample=p["oversample"], seed=0, max_restarts=10)
    for rep in range(2):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        loss = g.solve_loss(theta, M, bc, xt, **kw)
        loss.backward()
        e1.record(stream)
        torch.cuda.synchronize()
        theta.grad = None
        for c in bc:
            c.grad = None
    last = g.solve_loss.last
    out["differentiable_d12_n64"] = {
        "fp32_forward_plus_adjoint_seconds": e0.elapsed_time(e1) * 1e-3,
        "forward_iters": last["last_info"]["iters"],
        "adjoint_iters": last["last_adjoint_info"]["iters"],
        "forward_true_res": last["last_info"]["true_res"],
        "adjoint_true_res": last["last_adjoint_info"]["true_res"]}
    return out


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

    w, p = workload()
    # host oracle (rank 0, single GPU), one full solve, before any GPU work
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_full_solve(w, p)

    mode_name = args.mode or os.environ.get("TTSG_MODE", "tf32")
    mode = {"tf32": g.MODE_TF32, "fp32": g.MODE_FP32, "fp64": g.MODE_FP64,
            "bf16": g.MODE_BF16}[mode_name]
    op = g.op_to_device(w.op)
    b = g.TT.from_numpy(w.b)
    kw = dict(maxit=p["maxit"], tol=p["tol"], rmax=p["rmax"], s=p["s"], eta=p["eta"],
              stop_safety=0.1, r_sol=p["r_sol"], oversample=p["oversample"], seed=0,
              max_restarts=8, mode=mode)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    pk, pk_kind = peaks()
    alu = measured_alu_peaks(torch)

    ws = None
    for _ in range(args.warmup):
        x, info = g.tt_sgmres_solve(op, b, workspace=ws, **kw)
        if ws is None:
            ws = torch.empty(info["workspace_bytes"], dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    # headline: K whole solves, no per-launch profiling
    lib.tt_profile(0)
    clocks = Clocks(local)
    launches0 = lib.tt_launch_count()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    times, infos, x = timed_solves(torch, g, op, b, kw, ws, args.steps, flush, stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = lib.tt_launch_count() - launches0
    total_s = max_over_ranks(sum(times), "cuda")
    value = total_s / args.steps
    ms_per_step = value * 1e3
    info = infos[-1]
    iters = [i["iters"] for i in infos]

    # roofline: a separate pass of the same solves with every launch of every
    # kernel class bracketed by CUDA events on the solver's stream
    nprof = max(2, min(5, args.steps))
    lib.tt_profile(0xFF)
    ptimes, _, _ = timed_solves(torch, g, op, b, kw, ws, nprof, flush, stream)
    prof = read_profile(lib, ctypes)
    lib.tt_profile(0)
    prof_total_ms = sum(ptimes) * 1e3
    dom = max(prof, key=lambda k: prof[k]["ms"])
    v = prof[dom]
    avg_ms = v["ms"] / max(v["launches"], 1)
    fl_per = v["flops"] / max(v["launches"], 1)
    by_per = v["bytes"] / max(v["launches"], 1)
    if dom == "qr_f64":
        roof = {"bound": "alu", "achieved": fl_per / (avg_ms * 1e-3) / 1e12, "peak": alu["fp64"],
                "unit": "TFLOP/s", "peak_kind": "measured cuBLAS FP64 GEMM on this GPU",
                "flops_per_launch": fl_per,
                "flop_count": "2 m l^2 per m x l factorisation (the FP64 QR count 2 n l^3 with "
                              "m = n l)"}
    elif dom == "gemm":
        peak_c = alu["fp64"] if mode == g.MODE_FP64 else alu["fp32"]
        ai = fl_per / max(by_per, 1)
        if ai < peak_c * 1e12 / (pk["hbm_gbs"] * 1e9):
            roof = {"bound": "hbm", "achieved": by_per / (avg_ms * 1e-3) / 1e9,
                    "peak": pk["hbm_gbs"], "unit": "GB/s", "peak_kind": f"{pk_kind} copy bandwidth"}
        else:
            roof = {"bound": "alu", "achieved": fl_per / (avg_ms * 1e-3) / 1e12, "peak": peak_c,
                    "unit": "TFLOP/s", "peak_kind": "measured cuBLAS GEMM (no TF32) on this GPU"}
    else:
        roof = {"bound": "hbm", "achieved": by_per / (avg_ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "peak_kind": f"{pk_kind} copy bandwidth"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = TRAFFIC_BYTES.get(dom)
    roof["kernel"] = dom
    roof["launches_per_step"] = v["launches"] / nprof
    roof["avg_launch_us"] = avg_ms * 1e3
    roof["share_of_step"] = v["ms"] / prof_total_ms if prof_total_ms > 0 else None
    roof["timed_over"] = f"{nprof} event-profiled solves after the headline loop"

    # FP64 GPU leg (the "mixed vs FP64 GPU" comparison)
    fp64 = None
    if not args.no_fp64_leg and mode != g.MODE_FP64:
        kw64 = dict(kw, mode=g.MODE_FP64)
        xf, inf64 = g.tt_sgmres_solve(op, b, **kw64)
        ws64 = torch.empty(inf64["workspace_bytes"], dtype=torch.uint8, device="cuda")
        t64, i64, _ = timed_solves(torch, g, op, b, kw64, ws64, 2, flush, stream)
        fp64 = dict(seconds=statistics.median(t64), iters=i64[-1]["iters"],
                    true_res=i64[-1]["true_res"], cycles=i64[-1]["cycles"], runs=2)
        del ws64

    # end to end: pinned host inputs in, solution out, inside the timed interval
    op_h = [c.cpu().pin_memory() for c in op]
    b_h = [c.cpu().pin_memory() for c in b.cores]
    op_d = [torch.empty_like(c) for c in op]
    b_d = [torch.empty_like(c) for c in b.cores]
    h2d = sum(c.numel() * c.element_size() for c in op_h + b_h)
    e2e_s, d2h = [], 0
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for hsrc, ddst in zip(op_h + b_h, op_d + b_d):
            ddst.copy_(hsrc, non_blocking=True)
        xe, ie = g.tt_sgmres_solve(op_d, g.TT(b_d), workspace=ws, **kw)
        outs = [c.to("cpu", non_blocking=True) for c in xe.cores]
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_s.append(e0.elapsed_time(e1) * 1e-3)
        d2h = sum(o.numel() * o.element_size() for o in outs)
    e2e_value = max_over_ranks(sum(e2e_s), "cuda") / args.steps

    # the contraction half of the metric, from the profiled pass: algorithmic
    # TFLOP/s of the tcgen05 matvec (against the TF32 tensor peak; split TF32
    # issues three products per algorithmic one) and of the CUDA-core GEMMs
    contraction = {}
    for key, peak_c, kind in (("tc_matvec", pk["bf16_tflops_sustained"] * TF32_OVER_BF16,
                               f"{pk_kind} BF16 sustained x 1.1/2.25 (TF32 tensor)"),
                              ("gemm", alu["fp32"], "measured cuBLAS FP32 GEMM (no TF32)")):
        vv = prof[key]
        if vv["ms"] > 0 and vv["launches"] > 0:
            tf = vv["flops"] / (vv["ms"] * 1e-3) / 1e12
            contraction[key] = {"tflops": tf, "peak": peak_c, "frac": tf / peak_c,
                                "peak_kind": kind, "launches": vv["launches"],
                                "avg_launch_us": vv["ms"] * 1e3 / vv["launches"]}
    extras = None
    if not args.no_extras and world == 1:
        del ws
        torch.cuda.empty_cache()
        extras = extra_configs(torch, g, flush, stream,
                               [m for m in (mode_name, "fp64")])
    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"tf32": "tf32+f64", "bf16": "bf16+f64", "fp32": "f32+f64",
                      "fp64": "f64"}[mode_name],
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "mode": mode_name, "parallelism": "replicas",
                       "l2": "flushed (512 MiB write) before every step"},
            "iters_per_solve": statistics.median(iters), "true_res": info["true_res"],
            "svd_nonconverged": info.get("svd_nonconverged"),
            "cycles": info["cycles"], "max_rank": info["max_rank"],
            "gpu_launches": int(launches), "roofline": roof, "contraction": contraction,
            "measured_peaks_tflops": alu,
            "kernel_time_ms_by_class_profiled": {k: round(vv["ms"] / nprof, 3)
                                                 for k, vv in prof.items()},
            "e2e": {"value": e2e_value, "unit": "s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "clocks": clk}
    if fp64:
        line["fp64_gpu"] = fp64
        line["speedup_vs_fp64_gpu"] = fp64["seconds"] / value
    if cpu is not None:
        dt, cinfo = cpu
        line["cpu_baseline"] = {"value": dt, "unit": "s", "cores": host_cores(), "kind": "oracle",
                                "sample": f"1 full FP64 oracle solve ({cinfo['iters']} iterations, "
                                          f"{len(cinfo['cycles'])} cycle(s), true residual "
                                          f"{cinfo['true_res']:.2e}; restarts, final rounding and "
                                          f"exact residual included)"}
        line["speedup_vs_cpu_oracle"] = dt / value
    if extras:
        line["other_configs"] = extras
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_round_case(args):
    """One Gram-Schmidt rounding of the solver at a workload's sizes:
    ``Round(A v - h v)`` with v a random TT at the rank cap (d=10, n=64, rank
    64; or the large-rank d=20, n=128, rank 128), oversampling 10, tolerance
    1e-7, in the selected mode."""
    import torch
    import paper_2409_09471_gb300 as g
    mode_name = args.mode or "fp32"
    mode = {"tf32": g.MODE_TF32, "fp32": g.MODE_FP32, "fp64": g.MODE_FP64}[mode_name]
    if args.round_workload == "large_rank":
        w, r = ti.workload("large_rank"), 128
    else:
        (w, _), r = workload(), 64
    dt = g.mode_dtype(mode)
    v = g.TT.from_numpy(ti.random_tt(w.ns, [1] + [r] * (len(w.ns) - 1) + [1], seed=5), dt)
    Av = g.tt_matvec(g.op_to_device(w.op, dt), v, mode=mode)
    times = []
    for i in range(args.warmup + args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        y = g.tt_round_rand([Av, v], [1.0, -0.3], 1e-7, r, 10, seed=1, mode=mode)
        e1.record()
        torch.cuda.synchronize()
        if i >= args.warmup:
            times.append(e0.elapsed_time(e1))
    print(json.dumps({"case": "round", "workload": args.round_workload, "mode": mode_name,
                      "ms_per_call": statistics.median(times), "out_ranks": y.ranks[:4]}),
          flush=True)


def run_batched_case(args):
    """The batched workload: 64 right-hand sides (d=8, n=32 Laplacian, bond
    ranks U{1..12}, rank cap 150), solved by the library's worker pool in the
    selected mode (default FP32); one JSON line with the whole-batch time and
    RHS/s."""
    import torch
    import paper_2409_09471_gb300 as g
    mode_name = args.mode or "fp32"
    mode = {"tf32": g.MODE_TF32, "fp32": g.MODE_FP32, "fp64": g.MODE_FP64}[mode_name]
    w = ti.workload("batched")
    p = w.params
    op = g.op_to_device(w.op)
    bs = [g.TT.from_numpy(b) for b in w.b]
    kw = dict(maxit=p["maxit"], tol=p["tol"], rmax=p["rmax"], mode=mode, s=p["s"],
              round_tol=p["round_tol"], r_sol=p["r_sol"], oversample=p["oversample"],
              max_restarts=40, nworkers=args.workers)
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
