"""Benchmark: c-LSQR + Tikhonov/GCV through the C ABI on synthetic deblurring.

A step is one whole solve: itermax c-LSQR iterations (Algorithm 6) on one
observed tensor, then GCV on the projected bidiagonal and X_reg = V_k (*) y
(Algorithm 5's projection), all on the GPU, replayed as one CUDA graph.

Default workload (the precision form): a 512 x 512 x 64 video, frame k blurred
by its own Gaussian Toeplitz matrix (sigma 1.5 -> 3.5), noise 1e-3, 50
iterations, slice GEMMs in BF16 with FP32 accumulation; the FP32, TF32 and
FP32-level (BF16X3) forms run beside it, and the reported form must match the
FP32 form's reconstruction error within 2 %.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tcprod|reference]
                  [--workload video_512|two_sided_256|colour_64] [--precision ...]

Prints one JSON line (rank 0). Under torchrun each rank solves its own
replica (independent problems, no collective on the data path): "weak"
scaling, value = iterations/s summed over ranks (all ranks' iterations over
the slowest rank's time).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LSQR-c iters/s & solves/s at matched rel. error (BF16/TF32 vs FP32); % roofline"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0  # profiling recipe fallback (burst), used without MEASURED_PEAKS.json
# FP32 FFMA peak: 152 SMs x 128 FP32 lanes x 2 flop x clock (GB300 unit counts).
FP32_LANES = 152 * 128

WORKLOADS = {
    "two_sided_256": dict(kind="two_sided", n=256, n3=3, iters=50, seed=1),
    "colour_64": dict(kind="colour", n=64, n3=3, iters=30, seed=0),
    "video_512": dict(kind="video", n=512, n3=64, iters=50, seed=2),
}


# Iterations in one bounded oracle sample (about 10-30 s of host work).
CPU_SAMPLE = {"video_512": 2, "two_sided_256": 10, "colour_64": 30}


def make_problem(name):
    from paper_2103_11847_gb300 import inputs
    w = WORKLOADS[name]
    if w["kind"] == "two_sided":
        return inputs.two_sided_deblur(n=w["n"], n3=w["n3"], seed=w["seed"])
    if w["kind"] == "colour":
        return inputs.colour_deblur(n=w["n"], seed=w["seed"])
    return inputs.video_deblur(n=w["n"], frames=w["n3"], seed=w["seed"])


def product_flops(n1, n2, s, n3, two_sided):
    """Algorithmic flops of one c-product: the n3 slice GEMMs (the mode-3
    transforms are O(n3 log n3) per tube with a fast DCT and are not counted)."""
    f = 2.0 * n1 * n2 * s * n3
    if two_sided:
        f += 2.0 * n1 * s * s * n3
    return f


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 6:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[2 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------- CPU oracle ----

def oracle_problem(workload):
    """The workload's FP32 inputs as FP64 arrays and the oracle's operator:
    (op, adj, C) with C = op(X_true) + N formed by the oracle."""
    from oracle import cproduct as cp
    from paper_2103_11847_gb300 import inputs
    w = make_problem(workload)
    A = w["A"].astype(np.float32).astype(np.float64)
    B = w["B"].astype(np.float32).astype(np.float64) if w["B"] is not None else None
    op = lambda X: cp.cprod(A, X, B)
    adj = lambda Y: cp.cprod_adjoint(A, Y, B)
    C = inputs.scale_noise(op(w["X_true"]), w["G"], w["nu"]).astype(np.float32).astype(np.float64)
    return op, adj, C


def cpu_worker(workload, sample, steps, budget_s):
    """Time the FP64 oracle's c-LSQR on this host (run in a child process):
    `steps` runs of `sample` iterations from X_0 = 0 (each run includes the
    start-up product and norms, as a GPU solve does), stopping early once
    `budget_s` seconds have gone. Prints the per-run times and the CPU time
    the process used over them (its threads' user + system time)."""
    import resource
    from oracle import krylov as kr
    op, adj, C = oracle_problem(workload)
    times = []
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    for _ in range(steps):
        t = time.perf_counter()
        kr.lsqr(op, adj, C, itermax=sample)
        times.append(time.perf_counter() - t)
        if time.perf_counter() - t0 > budget_s:
            break
    wall = time.perf_counter() - t0
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    print(json.dumps({"times": times, "sample_iters": sample, "wall": wall, "cpu": cpu}))


def cpu_run(workload, sample, steps, budget_s, threads=None):
    """Run cpu_worker in a child process with `threads` BLAS/OpenMP threads
    (default: every core this process may run on)."""
    avail = len(os.sched_getaffinity(0))
    n = threads or avail
    env = dict(os.environ, OMP_NUM_THREADS=str(n), OPENBLAS_NUM_THREADS=str(n),
               MKL_NUM_THREADS=str(n), CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", workload,
                        "--cpu-sample", str(sample), "--cpu-steps", str(steps),
                        "--cpu-budget", str(budget_s)], capture_output=True, text=True, env=env,
                       timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(f"oracle worker failed: {r.stderr[-2000:]}")
    out = json.loads(r.stdout.strip().splitlines()[-1])
    out["threads_allowed"] = n
    out["cores_available"] = avail
    # cores the oracle kept busy: its CPU time over the wall time of the runs
    out["cores_used"] = max(1, int(round(out["cpu"] / max(out["wall"], 1e-9))))
    return out


def cpu_run_all_cores(workload, sample):
    """One single-threaded oracle worker per core this process may run on,
    all started together, each running the same bounded sample (independent
    replicas of the solve, as the GPU's replicas are): their times."""
    n = len(os.sched_getaffinity(0))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", workload, "--cpu-sample",
           str(sample), "--cpu-steps", "1", "--cpu-budget", "0"]
    t0 = time.perf_counter()
    procs = [subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                              env=env) for _ in range(n)]
    outs = [p.communicate(timeout=1800) for p in procs]
    wall = time.perf_counter() - t0
    if any(p.returncode != 0 for p in procs):
        raise RuntimeError("an oracle worker failed: " + next(e for (o, e), p in zip(outs, procs)
                                                          if p.returncode != 0)[-2000:])
    times = [json.loads(o.strip().splitlines()[-1])["times"][0] for o, _ in outs]
    return n, times, wall


def cpu_baseline(workload, sample=None):
    """The FP64 oracle as it stands on this host's cores: `sample` c-LSQR
    iterations of the workload (the bounded sample) by one process alone, then
    by one single-threaded process per core at once; iterations/s of the whole
    host (the all-core figure is the value, the one-core figure beside it)."""
    sample = sample or CPU_SAMPLE.get(workload, 2)
    out = cpu_run(workload, sample, 1, 0.0)
    t1 = out["times"][0]
    n, times, wall = cpu_run_all_cores(workload, sample)
    return {"value": n * sample / wall, "unit": "LSQR iterations/s", "cores": n,
            "cores_available": out["cores_available"], "kind": "oracle",
            "single_core": {"value": sample / t1, "cores": out["cores_used"], "seconds": t1},
            "sample": (f"c-LSQR runs of {sample} iterations from X_0 = 0 on the {workload} "
                       f"workload, start-up product and norms included (FP64 NumPy oracle): "
                       f"{n} single-threaded runs at once, one a core, {wall:.1f} s for all "
                       f"(slowest {max(times):.1f} s); one run alone {t1:.1f} s")}


# ---------------------------------------------------------------- GPU arm ----

def precision_forms(dev, peaks, steps=3):
    """The video workload (512 x 512 x 64, 50 c-LSQR iterations + Tikhonov/GCV)
    in FP32, TF32 and BF16 slice GEMMs: LSQR iterations/s, the reconstruction
    error of X_reg against the clean video (the matched-error check), and the
    transform-domain slice GEMM timed alone (tc_slice_gemm) against the HBM
    roofline: it reads A~ and X~ once and writes Y~ in FP32."""
    import torch
    from paper_2103_11847_gb300 import tcprod
    wl = WORKLOADS["video_512"]
    w = make_problem("video_512")
    n3, n1, n2 = w["A"].shape
    s = w["X_true"].shape[2]
    iters = wl["iters"]
    A = torch.from_numpy(w["A"].astype(np.float32)).to(dev)
    Xt = torch.from_numpy(w["X_true"].astype(np.float32)).to(dev)
    G = torch.from_numpy(w["G"].astype(np.float32)).to(dev)
    out = {"workload": f"video_512: c-LSQR {iters} it + Tikhonov/GCV, A {n1}x{n2}x{n3}, "
                       f"X {n2}x{s}x{n3}", "l2": "inputs (64-256 MB per tensor) exceed L2"}
    C = None
    st = torch.cuda.current_stream()
    for name, code in (("fp32", tcprod.TC_FP32), ("tf32", tcprod.TC_TF32), ("bf16", tcprod.TC_BF16),
                       ("bf16x3", tcprod.TC_BF16X3)):
        plan = tcprod.Plan(A, s=s, precision=code)
        if C is None:
            Cc = plan.cprod(Xt)
            C = (Cc + (w["nu"] * Cc.norm() / G.norm()) * G).contiguous()
        X = torch.empty(plan.xshape(), device=dev)
        Xr = torch.empty(plan.xshape(), device=dev)
        info = tcprod.new_info()
        tcprod.tc_lsqr_c(plan.handle, C, X, Xr, iters, 0.0, None, None, info)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            tcprod.tc_lsqr_c(plan.handle, C, X, Xr, iters, 0.0, None, None, info)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        inf = tcprod.read_info(info)
        # slice GEMM alone on a transform-domain operand of the plan's input type
        dt = torch.bfloat16 if name in ("bf16", "bf16x3") else torch.float32
        planes = 3 if name == "bf16x3" else 1
        Xh = torch.randn((planes * n3, n2, s), device=dev).to(dt)
        Yh = torch.empty((n3, n1, s), device=dev)
        for _ in range(3):
            tcprod.tc_slice_gemm(plan.handle, Xh, Yh)
        reps = 20
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(st)
        for _ in range(reps):
            tcprod.tc_slice_gemm(plan.handle, Xh, Yh)
        g1.record(st)
        torch.cuda.synchronize()
        gms = g0.elapsed_time(g1) / reps
        es = 2 * planes if name in ("bf16", "bf16x3") else 4
        gbytes = (n3 * n1 * n2 + n3 * n2 * s) * es + n3 * n1 * s * 4
        gflops = 2.0 * n1 * n2 * s * n3
        gbs = gbytes / (gms * 1e-3) / 1e9
        out[name] = {"iters_per_s": iters / (ms * 1e-3), "ms_per_solve": ms,
                     "rel_err_reg": float((Xr - Xt).norm() / Xt.norm()),
                     "rel_err_lsqr": float((X - Xt).norm() / Xt.norm()), "lambda": inf["lam"],
                     "status": inf["status"],
                     "slice_gemm": {"kernel": ("k_umma_gemm (tcgen05, six split-BF16 products)"
                                               if name == "bf16x3" else "k_umma_gemm (tcgen05)")
                                    if name != "fp32" else "k_slice_gemm (FFMA)", "ms": gms,
                                    "GB_per_s": gbs, "TFLOP_per_s": gflops / (gms * 1e-3) / 1e12,
                                    "hbm_frac": gbs / peaks.get("hbm_gbs", FALLBACK_HBM_GBS),
                                    "algorithmic_bytes": gbytes}}
        plan.close()
    out["bf16_dual"] = dual_route_form(A, C, Xt, s, iters, dev, peaks, steps)
    out["bf16_store"] = stored_products_form(A, C, Xt, s, iters, dev, steps)
    base = out["fp32"]["rel_err_reg"]
    for name in ("tf32", "bf16", "bf16x3", "bf16_dual", "bf16_store"):
        out[name]["matched_error"] = bool(abs(out[name]["rel_err_reg"] - base) <= 0.02 * base)
        out[name]["speedup_vs_fp32"] = out[name]["iters_per_s"] / out["fp32"]["iters_per_s"]
    # Algorithm 1's dct reading (ORTHODCT): off the fused route LSQR runs in the
    # transform domain (slice GEMMs + epilogue pass, no per-product transforms)
    od = {}
    for name, code in (("fp32", tcprod.TC_FP32), ("bf16", tcprod.TC_BF16)):
        plan = tcprod.Plan(A, s=s, precision=code, product=tcprod.TC_ORTHODCT)
        Cc = plan.cprod(Xt)
        Co = (Cc + (w["nu"] * Cc.norm() / G.norm()) * G).contiguous()
        X = torch.empty(plan.xshape(), device=dev)
        Xr = torch.empty(plan.xshape(), device=dev)
        info = tcprod.new_info()
        tcprod.tc_lsqr_c(plan.handle, Co, X, Xr, iters, 0.0, None, None, info)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            tcprod.tc_lsqr_c(plan.handle, Co, X, Xr, iters, 0.0, None, None, info)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        od[name] = {"iters_per_s": iters / (ms * 1e-3), "ms_per_solve": ms,
                    "rel_err_reg": float((Xr - Xt).norm() / Xt.norm())}
        plan.close()
    od["bf16"]["matched_error"] = bool(abs(od["bf16"]["rel_err_reg"] - od["fp32"]["rel_err_reg"])
                                       <= 0.02 * od["fp32"]["rel_err_reg"])
    out["orthodct_transform_domain"] = od
    return out


def stored_products_form(A, C, Xt, s, iters, dev, steps):
    """The BF16 form with its slice products stored in BF16 (TC_STORE_BF16):
    LSQR iterations/s and the reconstruction error (the headline's form)."""
    import torch
    from paper_2103_11847_gb300 import tcprod
    st = torch.cuda.current_stream()
    plan = tcprod.Plan(A, s=s, precision=tcprod.TC_BF16, store=tcprod.TC_STORE_BF16)
    X = torch.empty(plan.xshape(), device=dev)
    Xr = torch.empty(plan.xshape(), device=dev)
    info = tcprod.new_info()
    tcprod.tc_lsqr_c(plan.handle, C, X, Xr, iters, 0.0, None, None, info)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        tcprod.tc_lsqr_c(plan.handle, C, X, Xr, iters, 0.0, None, None, info)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    plan.close()
    return {"iters_per_s": iters / (ms * 1e-3), "ms_per_solve": ms,
            "rel_err_reg": float((Xr - Xt).norm() / Xt.norm()),
            "rel_err_lsqr": float((X - Xt).norm() / Xt.norm()),
            "store": "slice products rounded once to BF16 (TC_STORE_BF16), read back by the "
                     "BF16-input transform pass"}


def dual_route_form(A, C, Xt, s, iters, dev, peaks, steps):
    """The BF16 form on the dual-domain route (TC_ROUTE_DUAL): the solve's
    LSQR iterations/s and reconstruction error, and its two kernels timed
    alone against the HBM roofline. Per product: the tcgen05 GEMM with the
    Golub-Kahan update in its store (reads A~ and the operand in BF16 and prev
    in FP32, writes the FP32 result) and the change-of-domain pass (reads the
    FP32 result, writes the BF16 operand of the other product)."""
    import torch
    from paper_2103_11847_gb300 import tcprod
    n3, n1, n2 = A.shape
    st = torch.cuda.current_stream()
    plan = tcprod.Plan(A, s=s, precision=tcprod.TC_BF16, route=tcprod.TC_ROUTE_DUAL)
    X = torch.empty(plan.xshape(), device=dev)
    Xr = torch.empty(plan.xshape(), device=dev)
    info = tcprod.new_info()
    tcprod.tc_lsqr_c(plan.handle, C, X, Xr, iters, 0.0, None, None, info)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        tcprod.tc_lsqr_c(plan.handle, C, X, Xr, iters, 0.0, None, None, info)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    kernels = tcprod.tc_lsqr_graph_kernels(plan.handle)
    Xh = torch.randn((n3, n2, s), device=dev).to(torch.bfloat16)
    Y = torch.empty((n3, n1, s), device=dev)
    prev = torch.randn((n3, n1, s), device=dev)
    Yb = torch.empty((n3, n1, s), dtype=torch.bfloat16, device=dev)
    s0 = torch.tensor([2.0], dtype=torch.float64, device=dev)
    s1 = torch.tensor([3.0], dtype=torch.float64, device=dev)
    ss = torch.zeros(1, dtype=torch.float64, device=dev)
    hbm = peaks.get("hbm_gbs", FALLBACK_HBM_GBS)
    T = n3 * n1 * s
    gk_ms = graph_time(lambda: tcprod.tc_slice_gemm_gk(plan.handle, Xh, Y, s0, s1, prev), 30)
    gk_bytes = 2 * n3 * n1 * n2 + 2 * n3 * n2 * s + 8 * T
    du_ms = graph_time(lambda: tcprod.tc_transform_dual(plan.handle, tcprod.TC_DUAL_U, Y, Yb, ss),
                       30)
    du_bytes = 6 * T
    plan.close()
    k = lambda name, t, b: {"kernel": name, "ms": t, "GB_per_s": b / (t * 1e-3) / 1e9,
                            "hbm_frac": b / (t * 1e-3) / 1e9 / hbm, "algorithmic_bytes": b}
    return {"iters_per_s": iters / (ms * 1e-3), "ms_per_solve": ms,
            "rel_err_reg": float((Xr - Xt).norm() / Xt.norm()),
            "rel_err_lsqr": float((X - Xt).norm() / Xt.norm()),
            "kernels_per_solve": kernels,
            "route": "dual-domain (TC_ROUTE_DUAL): V x_3 M^-T and U x_3 M, one GEMM and one "
                     "change of domain a product",
            "gemm_gk": k("k_umma_gemm<EPI> (tcgen05, Golub-Kahan update in the store)", gk_ms,
                         gk_bytes),
            "change_of_domain": k("k_tube_tma<OUT_BF16, 2, NRM> (x_3 G, norm of x_3 M^-1)", du_ms,
                                  du_bytes)}


GROUP_TILES = {0: ["64x64 FFMA tiles of 4x4", "32x32 FFMA tiles of 4x2", "64x64 FFMA tiles of 8x4"],
               1: ["128x64 tcgen05 tiles", "128x128 tcgen05 tiles"]}


def group_form_text(code, grouped, tile, tune):
    if not grouped:
        return "one CUDA graph of per-problem child graphs"
    from paper_2103_11847_gb300 import tcprod
    names = GROUP_TILES[1 if code == tcprod.TC_BF16 else 0]
    timed = ", ".join("%s %.3f ms" % (nm, t) for nm, t in zip(names, tune))
    return ("grouped launches (one a phase for all problems, transforms fused into the "
            "products), %s picked by the autotuner (forward product: %s)" % (names[tile], timed))


def group_product_roofline(code, sizes, ms):
    """One grouped forward product of the batch (the autotuner's CUDA-event
    time of the chosen tile shape) against its roofline. Algorithmic bytes a
    problem: A~ (BF16 6 n^2, FP32 12 n^2) + the operand, prev and output
    (12 n^2 each); flops 2 n^3 a slice."""
    from paper_2103_11847_gb300 import tcprod
    peaks, src = load_peaks()
    sq = sum(n * n for n in sizes)
    cube = sum(n ** 3 for n in sizes)
    bf16 = code == tcprod.TC_BF16
    nbytes = (42 if bf16 else 48) * sq
    flops = 2.0 * 3 * cube
    gbs = nbytes / (ms * 1e-3) / 1e9
    hbm = peaks.get("hbm_gbs", FALLBACK_HBM_GBS)
    row = {"ms": ms, "algorithmic_bytes": nbytes, "flops": flops, "gb_s": gbs,
           "hbm_frac": gbs / hbm, "hbm_peak_source": f"MEASURED_PEAKS.json hbm_gbs ({src})",
           "tflops": flops / (ms * 1e-3) / 1e12}
    if bf16:
        row["traffic"] = captured_traffic("k_group_umma_bf16")
    else:
        fp = measured_peak("fp32_ffma_tflops")
        if fp:
            row["ffma_frac"] = row["tflops"] / fp
            row["ffma_peak_source"] = "profiles/peaks.json fp32_ffma_tflops (measured)"
    return row


def batched_form(dev, iters=40, count=128, steps=2):
    """128 independent colour deblurring problems of uneven sizes n in
    {64, 96, ..., 512} (n x n x 3, sigma ~ U[1, 4], noise ~ U[1e-4, 1e-2]),
    solved by c-LSQR (40 iterations) + Tikhonov/GCV in one graph launch, in FP32
    and BF16 slice GEMMs: solves/s and the mean reconstruction error."""
    import torch
    from paper_2103_11847_gb300 import inputs, tcprod
    sizes = inputs.batch_sizes(count)
    As, Cs, Xt = [], [], []
    for i, n in enumerate(sizes):
        w = inputs.batch_problem(i, n)
        A = torch.from_numpy(w["A"].astype(np.float32)).to(dev)
        As.append(A)
        Xt.append(torch.from_numpy(w["X_true"].astype(np.float32)).to(dev))
        Cs.append((w, A))
    out = {"workload": f"{count} problems n x n x 3, n in {{64..512}} (sum n^2 = "
                       f"{sum(n * n for n in sizes)}), c-LSQR {iters} it + Tikhonov/GCV",
           "launch": "one CUDA graph a batch (see each form)"}
    C_by_product = {}
    st = torch.cuda.current_stream()
    forms = (("fp32", tcprod.TC_FP32, tcprod.TC_TH), ("bf16", tcprod.TC_BF16, tcprod.TC_TH),
             ("fp32_orthodct", tcprod.TC_FP32, tcprod.TC_ORTHODCT),
             ("bf16_orthodct", tcprod.TC_BF16, tcprod.TC_ORTHODCT))
    for name, code, product in forms:
        h = tcprod.tc_batch_create(As, sizes, precision=code, product=product)
        if product not in C_by_product:  # C = A *c X + N, formed by the library's product
            C_dev = []
            for i, (w, A) in enumerate(Cs):
                p = tcprod.Plan(A, s=sizes[i], product=product)
                Cc = p.cprod(Xt[i])
                G = torch.from_numpy(w["G"].astype(np.float32)).to(dev)
                C_dev.append((Cc + (w["nu"] * Cc.norm() / G.norm()) * G).contiguous())
                p.close()
            C_by_product[product] = C_dev
        C_dev = C_by_product[product]
        Xs = [torch.empty_like(c) for c in C_dev]
        Xr = [torch.empty_like(c) for c in C_dev]
        infos = tcprod.new_infos(count)
        tcprod.tc_lsqr_c_batched(h, C_dev, Xs, Xr, iters, 0.0, None, infos)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            tcprod.tc_lsqr_c_batched(h, C_dev, Xs, Xr, iters, 0.0, None, infos)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        errs = [float((Xr[i] - Xt[i]).norm() / Xt[i].norm()) for i in range(count)]
        grouped, tile, tune = tcprod.tc_batch_info(h)
        out[name] = {"solves_per_s": count / (ms * 1e-3), "ms_per_batch": ms,
                     "iters_per_s": count * iters / (ms * 1e-3),
                     "mean_rel_err_reg": float(np.mean(errs)),
                     "form": group_form_text(code, grouped, tile, tune)}
        if grouped:
            out[name]["product_kernel"] = group_product_roofline(code, sizes, tune[tile])
        tcprod.tc_batch_destroy(h)
    base = out["fp32"]["mean_rel_err_reg"]
    out["bf16"]["matched_error"] = bool(abs(out["bf16"]["mean_rel_err_reg"] - base) <= 0.02 * base)
    # ORTHODCT is a different product (Algorithm 1's dct): matched against its own FP32
    bo = out["fp32_orthodct"]["mean_rel_err_reg"]
    out["bf16_orthodct"]["matched_error"] = bool(
        abs(out["bf16_orthodct"]["mean_rel_err_reg"] - bo) <= 0.02 * bo)
    out["bf16_orthodct"]["note"] = ("Algorithm 1's dct product; transform-domain iteration, "
                                    "epilogue in the tcgen05 GEMM")
    return out


def learned_form(train_count=10000):
    """Learned lambda / stop index: 10k c-LSQR solves (half the 20k of the
    full run, python -m paper_2103_11847_gb300.learn, to keep the default run
    near two minutes) labelled by
    tc_lsqr_label (128 x 128 x 3 and 256 x 256 x 3 images, every fifth a
    64 x 64 x 32 video; stopping indices up to 96), the network trained by
    tc_mlp_train, then the learned solve against plain GCV-driven c-LSQR (96
    steps, full GCV) on held-out 512 x 512 x 3 images and 512 x 512 x 32
    videos: with the 5% GCV fallback, and with the network's lambda alone."""
    from paper_2103_11847_gb300 import learn
    t0 = time.perf_counter()
    F, T = learn.training_data(train_count, sizes=[128, 256], video_every=5)
    t1 = time.perf_counter()
    mlp, hist = learn.train(F, T)
    t2 = time.perf_counter()
    k = T[:, 1].cpu().numpy()
    out = {"train": {"solves": train_count, "size": "128x128x3 / 256x256x3, every 5th 64x64x32",
                     "label_kmax": 96, "label_s": t1 - t0, "train_s": t2 - t1,
                     "label_k_mean": float(k.mean()), "label_k_std": float(k.std()),
                     "loss_first": float(hist[0].item()),
                     "loss_last50": float(hist[-50:].mean().item())},
           "gcv": "full (interior minimum) for the plain solve and the fallback check",
           "eval_512x512x3": learn.summarize(learn.compare(mlp, count=8)),
           "eval_512x512x3_network_lambda": learn.summarize(learn.compare(mlp, count=8,
                                                                          factor=1e30)),
           "eval_512x512x32": learn.summarize(learn.compare(mlp, count=2, frames=32))}
    mlp.close()
    return out


def source_digest(paths):
    """sha256 over the concatenated bytes of the given repository files."""
    import hashlib
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def captured_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu capture
    (profiles/traffic.json), or None once any source the kernel is built from
    no longer hashes to the captured version."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kernel)
        digest = source_digest(rec["sources"])
    except (OSError, ValueError, TypeError, KeyError):
        return None
    return rec["dram_bytes_per_launch"] if digest == rec["sha256"] else None


def graph_time(call, reps):
    """Device time of one call: `reps` back-to-back calls captured as one CUDA
    graph (no host launch overhead between them), replayed and timed with
    CUDA events on the replaying stream. The operands stay L2-resident between
    calls, as they do inside a solve."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(3):
            call()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for _ in range(reps):
            call()
    g.replay()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    g.replay()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


# Tables 1-4 (§4): image size, noise, and the iteration counts the paper used
# for DC-GMRES(10) (itermax), DC-GK (mmax, Tikhonov/GCV on the projected
# problem) and DC-LSQR (k_opt), with the paper's CPU seconds for context.
PAPER_TABLES = [
    (256, 1e-3, dict(gmres=(10, 5.21), gk=(15, 1.62), lsqr=(14, 1.23))),
    (256, 1e-2, dict(gmres=(15, 7.14), gk=(20, 1.92), lsqr=(15, 1.23))),
    (1024, 1e-3, dict(gmres=(10, 100.35), gk=(20, 25.33), lsqr=(15, 19.45))),
    (1024, 1e-2, dict(gmres=(15, 137.43), gk=(25, 30.22), lsqr=(20, 26.43))),
]


def paper_shaped(reps=3):
    """The paper's three methods on paper-shaped synthetic problems (the image
    sizes, blur and iteration counts of Tables 1-4; inputs.paper_deblur), each
    solve timed on the device (median of `reps` after a warm-up) with its
    relative error and SNR against the clean image."""
    import torch
    from paper_2103_11847_gb300 import inputs, tcprod
    dev = torch.device("cuda")
    st = torch.cuda.current_stream()
    rows = []
    for n, nu, methods in PAPER_TABLES:
        w = inputs.paper_deblur(n=n, nu=nu)
        A = torch.from_numpy(w["A"].astype(np.float32)).to(dev)
        B = torch.from_numpy(w["B"].astype(np.float32)).to(dev)
        Xt = torch.from_numpy(w["X_true"].astype(np.float32)).to(dev)
        G = torch.from_numpy(w["G"].astype(np.float32)).to(dev)
        plan = tcprod.Plan(A, B, s=n)
        Cc = plan.cprod(Xt)
        C = (Cc + (nu * Cc.norm() / G.norm()) * G).contiguous()
        X = torch.empty(plan.xshape(), device=dev)
        Xr = torch.empty(plan.xshape(), device=dev)
        info = tcprod.new_info()
        calls = {
            "DC-LSQR": (methods["lsqr"], lambda k: tcprod.tc_lsqr_c(plan.handle, C, X, None, k, 0.0,
                                                                    None, None, info), X),
            "DC-GK": (methods["gk"], lambda k: tcprod.tc_lsqr_c(plan.handle, C, X, Xr, k, 0.0, None,
                                                                None, info), Xr),
            "DC-GMRES(10)": (methods["gmres"], lambda k: tcprod.tc_gmres_c(plan.handle, C, None, X, 10,
                                                                          k, 0.0, None, info), X),
        }
        for name, ((k, paper_s), call, out) in calls.items():
            call(k)
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                call(k)
                e1.record(st)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            err = float((out - Xt).norm() / Xt.norm())
            snr = float(10.0 * torch.log10(((Xt - Xt.mean()) ** 2).sum() / ((out - Xt) ** 2).sum()))
            inf = tcprod.read_info(info)
            rows.append({"image": f"{n}x{n}x3", "nu": nu, "method": name, "iterations": k,
                         "gpu_ms": statistics.median(ts), "paper_cpu_s": paper_s,
                         "rel_err": err, "snr_db": snr, "lambda": inf["lam"]})
        plan.close()
    return rows


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, local, world


def replica_throughput(total_ms, steps, iters, world, device):
    """The slowest rank's timed region (max over ranks) and the whole-job value:
    the LSQR iterations every rank ran, over that time. Each rank solves its
    own problem (replicas), so this max is the only collective."""
    import torch
    t_max = float(total_ms)
    if world > 1:
        t = torch.tensor([t_max], device=device, dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_max = float(t.item())
    return t_max, world * steps * iters / (t_max / 1000.0)


def lsqr_floor_bytes(n1, n2, s, n3, precision, two_sided):
    """Algorithmic HBM bytes of one c-LSQR iteration on the fused schedule,
    2 T_A + 11 T: each product reads A~ (T_A, in the GEMM input type) and two
    tensors and writes one; the update reads X, W, V~ and writes X, W. T is
    one FP32 tensor of the larger of the two shapes."""
    T = 4.0 * max(n1, n2) * s * n3
    ea = {"fp32": 4, "tf32": 4, "bf16": 2, "bf16x3": 6}[precision]
    TA = ea * n1 * n2 * n3 + (ea * s * s * n3 if two_sided else 0)
    return 2 * TA + 11 * T


def effective_store(args, n3, two):
    """--store bf16 where the plan takes it (BF16, one-sided, 32 < n3 <= 64),
    else the FP32-stored products."""
    ok = args.precision == "bf16" and not two and 32 < n3 <= 64
    return "bf16" if (args.store == "bf16" and ok) else "f32"


def dominant_kernel(plan, args, dims, dev):
    """The kernel that takes the largest share of the workload's solve, as a
    callable that launches it once on the current stream with the operands
    it has inside the solve, and its algorithmic work per launch.

    * TF32/BF16/BF16X3 plans with n3 > 32: the tcgen05 transform pass back to
      the spatial domain with the Krylov epilogue (k_tube, FP32 out): it reads
      the slice-GEMM result and prev and writes the output (3 T bytes) and
      reduces its norm. Two launches an iteration.
    * FP32 plans with n3 <= 4: the fused product (k_cprod2 for the two-sided
      product with s <= 256, else k_fused_gemm), FFMA-bound.
    * Otherwise: the slice GEMMs of one product (tc_slice_gemm)."""
    import torch
    from paper_2103_11847_gb300 import tcprod
    n1, n2, s, n3, two = dims
    prec = args.precision
    if prec == "bf16" and n3 > 32 and getattr(args, "store", "f32") == "bf16" and not two:
        # BF16-stored slice products, chained passes: the pass back reads
        # them in BF16 (T/2), reads prev and writes the output (T each),
        # reduces the norm, and writes the next product's BF16 operand (T/2)
        P = n1 * s
        Yb = torch.randn((n3, n1, s), device=dev).to(torch.bfloat16)
        prev = torch.randn((n3, n1, s), device=dev)
        out = torch.empty((n3, n1, s), device=dev)
        nxt = torch.empty((n3, n1, s), dtype=torch.bfloat16, device=dev)
        ss = torch.zeros(1, dtype=torch.float64, device=dev)
        call = lambda: tcprod.tc_transform_bf16in(plan.handle, tcprod.TC_MINV, Yb, out, prev, ss,
                                                  which_next=tcprod.TC_MINVT, nxt=nxt)
        return dict(kernel="k_tube_chain (tcgen05 mode-3 transform M^-1 from the BF16 slice "
                           "products, Krylov epilogue and norm, and the next product's operand "
                           "x_3 M^-T in BF16)", call=call, bound="hbm",
                    work=(2.0 + 4.0 + 4.0 + 2.0) * n3 * P, traffic_key="k_tube_chain", reps=50)
    if prec != "fp32" and n3 > 32:
        P = n1 * s
        Yh = torch.randn((n3, n1, s), device=dev)
        prev = torch.randn((n3, n1, s), device=dev)
        out = torch.empty((n3, n1, s), device=dev)
        ss = torch.zeros(1, dtype=torch.float64, device=dev)
        name = ("k_tube<OUT_F32, 3> (tcgen05 mode-3 transform M^-1, three-plane split, with the "
                "Krylov epilogue and norm)" if prec == "bf16x3" else
                "k_tube<OUT_F32, 2> (tcgen05 mode-3 transform M^-1 with the Krylov epilogue "
                "and norm)")
        call = lambda: tcprod.tc_transform(plan.handle, tcprod.TC_MINV, Yh, out, prev, ss)
        return dict(kernel=name, call=call, bound="hbm", work=3 * 4.0 * n3 * P,
                    traffic_key="k_tube_f32", reps=50)
    fl = product_flops(n1, n2, s, n3, two)
    if two and prec != "fp32":  # the whole tensor-core product (two GEMMs and the passes)
        src = torch.randn((n3, n2, s), device=dev)
        dst = torch.empty((n3, n1, s), device=dev)
        return dict(kernel=f"two-sided tensor-core product ({prec}: transform, two tcgen05 "
                           "GEMMs, transform back)",
                    call=lambda: tcprod.tc_cprod(plan.handle, src, dst), bound="tensor",
                    work=fl, precision=prec, traffic_key=None, reps=100)
    if n3 <= 4 and prec == "fp32":
        src = torch.randn((n3, n2, s), device=dev)
        dst = torch.empty((n3, n1, s), device=dev)
        name = ("k_cprod2 (the whole two-sided product, one launch)" if two and s <= 256
                else "k_fused_gemm (the GEMM stages of one c-product)")
        return dict(kernel=name, call=lambda: tcprod.tc_cprod(plan.handle, src, dst), bound="alu",
                    work=fl, traffic_key="k_cprod2" if two and s <= 256 else None, reps=200)
    lowp_dt = torch.bfloat16 if prec in ("bf16", "bf16x3") else torch.float32
    planes = 3 if prec == "bf16x3" else 1
    src = torch.randn((planes * n3, n2, s), device=dev).to(lowp_dt)
    dst = torch.empty((n3, n1, s), device=dev)
    name = ("k_umma_gemm (tcgen05 slice GEMMs of one product"
            + (", six split-BF16 products)" if planes == 3 else ")")
            if prec != "fp32" else "k_slice_gemm (FFMA slice GEMMs of one product)")
    es = {"bf16": 2, "bf16x3": 6}.get(prec, 4)
    bound = {"bf16x3": "tensor", "fp32": "alu"}.get(prec, "hbm")
    return dict(kernel=name, call=lambda: tcprod.tc_slice_gemm(plan.handle, src, dst),
                bound=bound, flops=fl,
                work=fl if bound != "hbm" else (n3 * n1 * n2 + n3 * n2 * s) * es + n3 * n1 * s * 4,
                traffic_key=None, reps=50)


def roofline_line(dk, ms, peaks, src_peaks):
    """roofline object of the JSON line for the dominant kernel `dk` whose
    average launch took `ms` milliseconds."""
    if dk["bound"] == "hbm":
        peak = peaks.get("hbm_gbs", FALLBACK_HBM_GBS)
        ach = dk["work"] / (ms * 1e-3) / 1e9
        unit, psrc = "GB/s", f"MEASURED_PEAKS.json hbm_gbs ({src_peaks}, burst copy)"
        extra = {"algorithmic_bytes": dk["work"]}
    elif dk["bound"] == "tensor":
        # FP32-level (BF16X3): six BF16 products per product; TF32 runs at half
        # the BF16 rate (the recipe's nominal ratio); BF16 at the BF16 rate
        prec = dk.get("precision", "bf16x3")
        tf = measured_peak("tf32_mma_tflops") if prec == "tf32" else None
        if tf is not None:
            peak, psrc = tf, "profiles/peaks.json tf32_mma_tflops (measured tcgen05 TF32 rate)"
        else:
            div = {"bf16x3": 6.0, "tf32": 2.0, "bf16": 1.0}[prec]
            peak = peaks.get("bf16_tflops", FALLBACK_BF16_TFLOPS) / div
            psrc = f"MEASURED_PEAKS.json bf16_tflops ({src_peaks}) / {div:g}"
        ach = dk["work"] / (ms * 1e-3) / 1e12
        unit = "TFLOP/s"
        extra = {"algorithmic_flops": dk["work"]}
    else:
        fp = measured_peak("fp32_ffma_tflops")
        if fp is not None:
            peak, psrc = fp, "profiles/peaks.json fp32_ffma_tflops (measured FFMA loop)"
        else:
            sm_max = peaks.get("sm_max_mhz", 2070.0)
            peak = FP32_LANES * 2 * sm_max * 1e6 / 1e12
            psrc = f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (unit count x max clock)"
        ach = dk["work"] / (ms * 1e-3) / 1e12
        unit = "TFLOP/s"
        extra = {"algorithmic_flops": dk["work"]}
    traffic = captured_traffic(dk["traffic_key"]) if dk.get("traffic_key") else None
    r = {"kernel": dk["kernel"], "bound": dk["bound"], "achieved": ach, "peak": peak,
         "unit": unit, "frac": ach / peak, "traffic": traffic, "peak_source": psrc,
         "launch_ms": ms}
    r.update(extra)
    return r


def measured_peak(key):
    """A peak this repository measured (profiles/peaks.json), or None."""
    try:
        with open(os.path.join(ROOT, "profiles", "peaks.json")) as f:
            return float(json.load(f)[key])
    except (OSError, ValueError, KeyError, TypeError):
        return None


def run_gpu(args):
    import torch
    from paper_2103_11847_gb300 import tcprod

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    wl = WORKLOADS[args.workload]
    w = make_problem(args.workload)
    n3, n1, n2 = w["A"].shape
    two = w["B"] is not None
    s = w["B"].shape[1] if two else w["X_true"].shape[2]
    iters = args.iters or wl["iters"]
    dev = torch.device("cuda", local)
    A = torch.from_numpy(w["A"].astype(np.float32)).to(dev)
    B = torch.from_numpy(w["B"].astype(np.float32)).to(dev) if two else None
    Xt = torch.from_numpy(w["X_true"].astype(np.float32)).to(dev)
    G = torch.from_numpy(w["G"].astype(np.float32)).to(dev)
    prec = {"fp32": tcprod.TC_FP32, "tf32": tcprod.TC_TF32, "bf16": tcprod.TC_BF16,
            "bf16x3": tcprod.TC_BF16X3}[args.precision]
    product = {"th": tcprod.TC_TH, "orthodct": tcprod.TC_ORTHODCT}[args.product]
    route = {"auto": tcprod.TC_ROUTE_AUTO, "spatial": tcprod.TC_ROUTE_SPATIAL,
             "dual": tcprod.TC_ROUTE_DUAL}[args.route]
    args.store = effective_store(args, n3, two)
    store = {"f32": tcprod.TC_STORE_F32, "bf16": tcprod.TC_STORE_BF16}[args.store]
    plan = tcprod.Plan(A, B, s=s, precision=prec, product=product, route=route, store=store)
    # observation C = M(X_true) + N with ||N|| = nu ||M(X_true)||, formed on the GPU
    Cc = plan.cprod(Xt)
    C = (Cc + (w["nu"] * Cc.norm() / G.norm()) * G).contiguous()
    X = torch.empty(plan.xshape(), device=dev)
    Xr = torch.empty(plan.xshape(), device=dev)
    info = tcprod.new_info()
    st = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def solve():
        tcprod.tc_lsqr_c(plan.handle, C, X, Xr, iters, 0.0, None, None, info)

    for _ in range(max(args.warmup, 3)):
        solve()
    torch.cuda.synchronize()
    kernels_per_solve = tcprod.tc_lsqr_graph_kernels(plan.handle)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        flush.zero_()  # evict the L2 between timed steps (outside the events)
        starts[i].record(st)
        solve()
        ends[i].record(st)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = sum(step_ms)

    # the dominant kernel alone, on the stream it is launched on, with the
    # operands it has inside the solve (back-to-back launches, CUDA events)
    dk = dominant_kernel(plan, args, (n1, n2, s, n3, two), dev)
    dk_ms = graph_time(dk["call"], dk["reps"])
    clk = clocks.stop()

    # end to end through the public API: pinned host C in, X_reg out, every step
    C_host = C.cpu().pin_memory()
    Xr_host = torch.empty(plan.xshape(), dtype=torch.float32).pin_memory()
    info_host = torch.empty(info.numel(), dtype=torch.uint8).pin_memory()
    Cdev = torch.empty_like(C)
    ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    ee0.record(st)
    for _ in range(e2e_steps):
        Cdev.copy_(C_host, non_blocking=True)
        tcprod.tc_lsqr_c(plan.handle, Cdev, X, Xr, iters, 0.0, None, None, info)
        Xr_host.copy_(Xr, non_blocking=True)
        info_host.copy_(info, non_blocking=True)
    ee1.record(st)
    torch.cuda.synchronize()
    e2e_ms = ee0.elapsed_time(ee1) / e2e_steps
    tcprod.tc_lsqr_c(plan.handle, C, X, Xr, iters, 0.0, None, None, info)  # the solve reported
    inf = tcprod.read_info(info)
    if tcprod.tc_plan_status(plan.handle) != tcprod.TC_OK:
        raise RuntimeError("a bounded wait of a tensor-core kernel gave up during the bench")

    t_max, value = replica_throughput(total_ms, args.steps, iters, world, dev)
    if rank == 0:
        peaks, src_peaks = load_peaks()
        hbm = peaks.get("hbm_gbs", FALLBACK_HBM_GBS)
        ms_iter = t_max / args.steps / iters
        floor_b = lsqr_floor_bytes(n1, n2, s, n3, args.precision, two)
        line = {
            "metric": METRIC, "value": value, "unit": "LSQR iterations/s",
            "solves_per_s": value / iters, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16x3": "f32-level: three BF16 planes an operand, six "
                      "products, f32 accumulate"}.get(args.precision,
                                                       f"{args.precision} GEMM inputs, f32")
            + (" (slice products stored in bf16)" if args.store == "bf16" else ""),
            "data": "synthetic (seeded video/image + Gaussian Toeplitz blurs + 1e-3 noise)",
            "config": {"workload": WORKLOAD_NAMES[args.workload].format(
                           iters=iters, n1=n1, n2=n2, n3=n3, s=s),
                       "precision": args.precision, "product": args.product,
                       "store": args.store,
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline_line(dk, dk_ms, peaks, src_peaks),
            "solve_roofline": {
                "bytes_per_iteration": floor_b,
                "floor_us_per_iteration": floor_b / (hbm * 1e9) * 1e6,
                "measured_us_per_iteration": ms_iter * 1e3,
                "solve_frac": floor_b / (hbm * 1e9) / (ms_iter * 1e-3),
                "definition": "algorithmic bytes 2 T_A + 11 T per c-LSQR iteration at the "
                              "measured HBM copy rate, over the measured time per iteration "
                              "of the whole solve (start-up, GCV and X_reg included)"},
            "e2e": {"value": iters / (e2e_ms / 1000.0) * world, "unit": "LSQR iterations/s",
                    "h2d_bytes_per_step": int(C.numel() * 4),
                    "d2h_bytes_per_step": int(Xr.numel() * 4 + info.numel())},
            "gpu_launches": args.steps * kernels_per_solve,
            "gpu_launches_per_solve": kernels_per_solve,
            "clocks": clk,
            "solve": {"iters": inf["iters"], "status": inf["status"], "lambda": inf["lam"],
                      "resid": inf["resid"],
                      "rel_err_reg": float((Xr - Xt).norm() / Xt.norm()),
                      "rel_err_lsqr": float((X - Xt).norm() / Xt.norm())},
        }
        plan.close()
        if not args.no_precision_forms and world == 1:
            if args.workload == "video_512":
                pf = precision_forms(dev, peaks)
                line["precision_forms"] = pf
                form = "bf16_store" if args.store == "bf16" else args.precision
                if form in pf:
                    line["matched_error"] = {
                        "form": form, "rel_err_reg": pf[form]["rel_err_reg"],
                        "fp32_rel_err_reg": pf["fp32"]["rel_err_reg"],
                        "matched": pf[form].get("matched_error", True),
                        "rule": "|e - e_fp32| <= 0.02 e_fp32 on X_reg vs the clean video",
                        "speedup_vs_fp32": value / pf["fp32"]["iters_per_s"]}
            line["two_sided_256"] = two_sided_form(dev, peaks, src_peaks)
            line["batched_form"] = batched_form(dev)
            line["learned_form"] = learned_form()
            line["paper_shaped"] = paper_shaped()
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(line), flush=True)
    else:
        plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def two_sided_form(dev, peaks, src_peaks, steps=10):
    """The two-sided 256 x 256 x 3 workload (A *c X *c B, 50 c-LSQR iterations
    + Tikhonov/GCV): FP32 (the fused one-launch FFMA product) and the
    tensor-core forms (BF16X3 at FP32 level, TF32), iterations/s, the
    reconstruction error, and the FP32 product's roofline."""
    import torch
    from paper_2103_11847_gb300 import tcprod
    w = make_problem("two_sided_256")
    n3, n1, n2 = w["A"].shape
    s = w["B"].shape[1]
    iters = WORKLOADS["two_sided_256"]["iters"]
    A = torch.from_numpy(w["A"].astype(np.float32)).to(dev)
    B = torch.from_numpy(w["B"].astype(np.float32)).to(dev)
    Xt = torch.from_numpy(w["X_true"].astype(np.float32)).to(dev)
    G = torch.from_numpy(w["G"].astype(np.float32)).to(dev)
    st = torch.cuda.current_stream()
    out = {"workload": WORKLOAD_NAMES["two_sided_256"].format(iters=iters, n1=n1, n2=n2, n3=n3,
                                                               s=s)}
    C = None
    for name, code in (("fp32", tcprod.TC_FP32), ("bf16x3", tcprod.TC_BF16X3),
                       ("tf32", tcprod.TC_TF32)):
        plan = tcprod.Plan(A, B, s=s, precision=code)
        if C is None:
            Cc = plan.cprod(Xt)
            C = (Cc + (w["nu"] * Cc.norm() / G.norm()) * G).contiguous()
        X = torch.empty(plan.xshape(), device=dev)
        Xr = torch.empty(plan.xshape(), device=dev)
        info = tcprod.new_info()
        for _ in range(3):
            tcprod.tc_lsqr_c(plan.handle, C, X, Xr, iters, 0.0, None, None, info)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            tcprod.tc_lsqr_c(plan.handle, C, X, Xr, iters, 0.0, None, None, info)
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        r = {"iters_per_s": iters / (ms * 1e-3), "ms_per_solve": ms,
             "rel_err_reg": float((Xr - Xt).norm() / Xt.norm()),
             "launches_per_solve": tcprod.tc_lsqr_graph_kernels(plan.handle)}
        # one whole product alone (every launch of it), back to back
        src, dst = torch.randn(plan.xshape(), device=dev), torch.empty(plan.yshape(), device=dev)
        pms = graph_time(lambda: tcprod.tc_cprod(plan.handle, src, dst), 100)
        r["product_us"] = pms * 1e3
        if name == "fp32":
            class _A:
                precision = "fp32"
            dk = dominant_kernel(plan, _A, (n1, n2, s, n3, True), dev)
            r["roofline"] = roofline_line(dk, graph_time(dk["call"], dk["reps"]), peaks, src_peaks)
        else:  # FP32-level products: six BF16 products each (BF16X3), or TF32 rate
            fl = product_flops(n1, n2, s, n3, True)
            r["product_tflops"] = fl / (pms * 1e-3) / 1e12
        out[name] = r
        plan.close()
    base = out["fp32"]["rel_err_reg"]
    for name in ("bf16x3", "tf32"):
        out[name]["matched_error"] = bool(abs(out[name]["rel_err_reg"] - base) <= 0.02 * base)
    return out


WORKLOAD_NAMES = {
    "video_512": ("video_512: c-LSQR {iters} it + Tikhonov/GCV on a {n1}x{n2}x{n3} video "
                  "(A {n1}x{n2}x{n3}, frame k blurred by G(sigma_k), sigma 1.5 -> 3.5; "
                  "X {n2}x{s}x{n3})"),
    "two_sided_256": ("two_sided_256: c-LSQR {iters} it + Tikhonov/GCV, A *c X *c B with "
                      "A {n1}x{n2}x{n3}, B {s}x{s}x{n3}, X {n2}x{s}x{n3}"),
    "colour_64": ("colour_64: c-LSQR {iters} it + Tikhonov/GCV, A {n1}x{n2}x{n3}, "
                  "X {n2}x{s}x{n3}"),
}


def run_reference(args):
    """The oracle as the reference arm, on all the host's cores: each step
    one bounded sample of the workload (CPU_SAMPLE iterations from X_0 = 0)
    by one single-threaded run a core, all started together (the oracle's
    einsums use one core each); value = the iterations of all runs over the
    steps' wall time. The run stops early, after at least two steps, once
    about two minutes have gone."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    sample = CPU_SAMPLE.get(args.workload, 2)
    t0 = time.perf_counter()
    walls, runs, cores = [], 0, 1
    for step in range(max(args.steps, 1)):
        cores, times, wall = cpu_run_all_cores(args.workload, sample)
        walls.append(wall)
        runs += len(times)
        if step >= 1 and time.perf_counter() - t0 > args.ref_budget:
            break
    el = time.perf_counter() - t0
    value = sample * runs / sum(walls)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "LSQR iterations/s",
        "n_gpus": world, "steps": len(walls), "steps_requested": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": 1000.0 * sum(walls) / len(walls),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded video/image + Gaussian Toeplitz blurs + 1e-3 noise)",
        "config": {"workload": f"{args.workload}: c-LSQR (FP64 NumPy oracle on the host cores); "
                               f"each step a bounded sample of {sample} iterations of the "
                               f"{wl['iters']}-iteration solve, one single-threaded run a "
                               f"core",
                   "wall_s": el},
        "cpu_baseline": {"kind": "oracle", "cores": cores,
                         "cores_available": len(os.sched_getaffinity(0)), "value": value,
                         "unit": "LSQR iterations/s",
                         "sample": f"{len(walls)} steps of {cores} concurrent runs of {sample} "
                                   f"c-LSQR iterations from X_0 = 0 (start-up product and "
                                   f"norms included, process start included), "
                                   f"{sum(walls):.1f} s"},
        "e2e": {"value": value, "unit": "LSQR iterations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="tcprod", choices=["tcprod", "reference"])
    ap.add_argument("--workload", default="video_512", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision-forms", action="store_true",
                    help="only the main workload (no other forms, batch, learned, two-sided)")
    ap.add_argument("--iters", type=int, default=0, help="override the workload's iterations")
    ap.add_argument("--precision", default=None, choices=["fp32", "tf32", "bf16", "bf16x3"],
                    help="slice-GEMM inputs of the main workload (default: bf16 for video_512, "
                         "fp32 otherwise)")
    ap.add_argument("--store", default="bf16", choices=["f32", "bf16"],
                    help="how the BF16 slice products reach the transform back (tc_store; "
                    "bf16 applies to BF16 one-sided plans with 32 < n3 <= 64)")
    ap.add_argument("--route", default="auto", choices=["auto", "spatial", "dual"],
                    help="where c-LSQR keeps its vectors (tc_route)")
    ap.add_argument("--product", default="th", choices=["th", "orthodct"],
                    help="c-product reading: Definition 2.1 (th) or Algorithm 1's dct "
                         "(orthodct; off the fused route LSQR then runs in the transform domain)")
    ap.add_argument("--paper-shaped", action="store_true",
                    help="time the paper's three methods on the shapes of its Tables 1-4")
    ap.add_argument("--kernel-only", action="store_true",
                    help="launch only the workload's dominant kernel (8 launches) and then 4 "
                         "whole c-products, for profiling captures")
    ap.add_argument("--batched", action="store_true",
                    help="run only the batched form (128 problems, every precision form) and "
                         "print its JSON, for profiling captures")
    ap.add_argument("--ref-budget", type=float, default=120.0,
                    help="seconds after which the reference arm stops taking steps")
    ap.add_argument("--cpu-worker", default=None)
    ap.add_argument("--cpu-sample", type=int, default=2)
    ap.add_argument("--cpu-steps", type=int, default=1)
    ap.add_argument("--cpu-budget", type=float, default=0.0)
    args = ap.parse_args()
    if args.precision is None:
        args.precision = "bf16" if args.workload == "video_512" else "fp32"
    if args.cpu_worker:
        cpu_worker(args.cpu_worker, args.cpu_sample, args.cpu_steps, args.cpu_budget)
        return
    if args.paper_shaped:
        for row in paper_shaped():
            print(json.dumps(row))
        return
    if args.kernel_only:
        kernel_only(args)
        return
    if args.batched:
        print(json.dumps(batched_form("cuda")))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


def kernel_only(args):
    """Plan the workload, launch its dominant kernel 8 times and then 4 whole
    c-products (the command profiling captures run)."""
    import torch
    from paper_2103_11847_gb300 import tcprod
    w = make_problem(args.workload)
    n3, n1, n2 = w["A"].shape
    two = w["B"] is not None
    s = w["B"].shape[1] if two else w["X_true"].shape[2]
    dev = torch.device("cuda", 0)
    A = torch.from_numpy(w["A"].astype(np.float32)).to(dev)
    B = torch.from_numpy(w["B"].astype(np.float32)).to(dev) if two else None
    prec = {"fp32": tcprod.TC_FP32, "tf32": tcprod.TC_TF32, "bf16": tcprod.TC_BF16,
            "bf16x3": tcprod.TC_BF16X3}[args.precision]
    route = {"auto": tcprod.TC_ROUTE_AUTO, "spatial": tcprod.TC_ROUTE_SPATIAL,
             "dual": tcprod.TC_ROUTE_DUAL}[args.route]
    args.store = effective_store(args, n3, two)
    store = {"f32": tcprod.TC_STORE_F32, "bf16": tcprod.TC_STORE_BF16}[args.store]
    plan = tcprod.Plan(A, B, s=s, precision=prec, route=route, store=store)
    dk = dominant_kernel(plan, args, (n1, n2, s, n3, two), dev)
    for _ in range(8):
        dk["call"]()
    if route == tcprod.TC_ROUTE_DUAL:
        # the dual-domain route's two kernels, four launches each: the GEMM
        # with the Golub-Kahan update, then the change of domain
        Xh = torch.randn((n3, n2, s), device=dev).to(torch.bfloat16)
        Y = torch.empty((n3, n1, s), device=dev)
        prev = torch.randn((n3, n1, s), device=dev)
        Yb = torch.empty((n3, n1, s), dtype=torch.bfloat16, device=dev)
        s0 = torch.tensor([2.0], dtype=torch.float64, device=dev)
        s1 = torch.tensor([3.0], dtype=torch.float64, device=dev)
        ss = torch.zeros(1, dtype=torch.float64, device=dev)
        for _ in range(4):
            tcprod.tc_slice_gemm_gk(plan.handle, Xh, Y, s0, s1, prev)
        for _ in range(4):
            tcprod.tc_transform_dual(plan.handle, tcprod.TC_DUAL_U, Y, Yb, ss)
    # then whole forward products (every pass of one product, e.g. the
    # transform to the GEMM operand before the slice GEMMs)
    Xp, Yp = torch.randn(plan.xshape(), device=dev), torch.empty(plan.yshape(), device=dev)
    for _ in range(4):
        tcprod.tc_cprod(plan.handle, Xp, Yp)
    torch.cuda.synchronize()
    status = tcprod.tc_plan_status(plan.handle)
    plan.close()
    print(json.dumps({"kernel": dk["kernel"], "launches": 8, "products": 4, "status": status}))
    if status != tcprod.TC_OK:
        sys.exit(1)


if __name__ == "__main__":
    main()
