"""Benchmark: c-LSQR + Tikhonov/GCV through the C ABI on synthetic deblurring.

A step is one whole solve: itermax c-LSQR iterations (Algorithm 6) on one
observed tensor, then GCV on the projected bidiagonal and X_reg = V_k (*) y
(Algorithm 5's projection), all on the GPU, replayed as one CUDA graph.

Default workload: two-sided A *c X *c B, 256 x 256 x 3, Gaussian blurs
(sigma 3 and 2, half-band 8), noise 1e-3, 50 iterations.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl tcprod|reference]
                  [--workload two_sided_256|colour_64|video_512]

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


def lsqr_kernel_launches(iters, two_sided, fused, keep_basis=True, precision="fp32", s=0, n3=64):
    """Kernels one solve launches (mirrors the schedule in csrc/solvers.cu).
    A fused product is one launch, except two-sided with s > 256 (two)."""
    if fused:
        per_product = 2 if (two_sided and s > 256) else 1
    else:
        per_product = 4 if two_sided else 3
    if precision != "fp32":  # transform, [transpose for TF32], tcgen05 GEMM, transform back
        per_product = 4 if precision == "tf32" else 3
        if precision == "bf16x3" and n3 <= 32:  # FP32 transform pass, then the three planes
            per_product = 4
    init = 1 + per_product + 1 + (1 if keep_basis else 0) + 1
    # product, adjoint, and the LSQR step: inside the next product on the
    # two-sided fused route (s <= 256), else its own launch; the last step
    # always has its own launch
    inside = fused and two_sided and s <= 256 and precision == "fp32"
    per_iter = 2 * per_product + (0 if inside else 1)
    tail = (1 if inside else 0) + (5 if keep_basis else 0) + 1  # GCV levels, final, combine; info
    return init + iters * per_iter + tail


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

def cpu_worker(workload, budget_s):
    """Time the FP64 oracle's c-LSQR on this host (run in a child process)."""
    from oracle import cproduct as cp
    from oracle import krylov as kr
    from paper_2103_11847_gb300 import inputs
    w = make_problem(workload)
    A = w["A"].astype(np.float32).astype(np.float64)
    B = w["B"].astype(np.float32).astype(np.float64) if w["B"] is not None else None
    op = lambda X: cp.cprod(A, X, B)
    adj = lambda Y: cp.cprod_adjoint(A, Y, B)
    C = inputs.scale_noise(op(w["X_true"]), w["G"], w["nu"]).astype(np.float32).astype(np.float64)
    iters = WORKLOADS[workload]["iters"]
    sample = max(2, min(iters, 10))
    kr.lsqr(op, adj, C, itermax=2)  # warm-up
    done, t0 = 0, time.perf_counter()
    while True:
        kr.lsqr(op, adj, C, itermax=sample)
        done += sample
        el = time.perf_counter() - t0
        if el > budget_s:
            break
    print(json.dumps({"iters": done, "seconds": el, "sample_iters": sample}))


def cpu_baseline(workload, budget_s=12.0):
    cores = len(os.sched_getaffinity(0))
    env = dict(os.environ, OMP_NUM_THREADS=str(cores), OPENBLAS_NUM_THREADS=str(cores),
               MKL_NUM_THREADS=str(cores), CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", workload,
                        "--cpu-budget", str(budget_s)], capture_output=True, text=True, env=env,
                       timeout=600)
    out = json.loads(r.stdout.strip().splitlines()[-1])
    value = out["iters"] / out["seconds"]
    return {"value": value, "unit": "LSQR iterations/s", "cores": cores, "kind": "oracle",
            "sample": (f"{out['iters']} c-LSQR iterations of the {workload} workload in runs of "
                       f"{out['sample_iters']} (FP64 NumPy oracle, {out['seconds']:.1f} s)")}


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
    base = out["fp32"]["rel_err_reg"]
    for name in ("tf32", "bf16", "bf16x3"):
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
           "launch": "one CUDA graph of per-problem child graphs"}
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
        out[name] = {"solves_per_s": count / (ms * 1e-3), "ms_per_batch": ms,
                     "iters_per_s": count * iters / (ms * 1e-3),
                     "mean_rel_err_reg": float(np.mean(errs))}
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


def learned_form(train_count=20000):
    """Learned lambda / stop index: 20k c-LSQR solves of 128 x 128 x 3 problems
    labelled by tc_lsqr_label, the network trained by tc_mlp_train, then the
    learned solve against plain GCV-driven c-LSQR (40 steps) on held-out
    512 x 512 x 3 images and a 512 x 512 x 32 video."""
    import torch
    from paper_2103_11847_gb300 import learn
    t0 = time.perf_counter()
    F, T = learn.training_data(train_count)
    t1 = time.perf_counter()
    mlp, hist = learn.train(F, T)
    t2 = time.perf_counter()
    out = {"train": {"solves": train_count, "size": "128x128x3", "label_s": t1 - t0,
                     "train_s": t2 - t1, "loss_first": float(hist[0].item()),
                     "loss_last50": float(hist[-50:].mean().item())},
           "eval_512x512x3": learn.summarize(learn.compare(mlp, count=8)),
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
    plan = tcprod.Plan(A, B, s=s, precision=prec, product=product)
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

    # dominant kernel, timed alone on the stream. n3 <= 4 (FP32): the fused
    # product launches (one for the two-sided product with s <= 256), timed
    # through tc_cprod. Otherwise: the slice GEMMs of one product (tc_slice_gemm).
    fl = product_flops(n1, n2, s, n3, two)
    reps = 200
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if n3 <= 4 and args.precision == "fp32":
        roof_kernel = ("k_cprod2 (the whole two-sided product, one launch)" if two and s <= 256
                       else "k_fused_gemm (the GEMM stages of one c-product)")
        src, dst = Xr, torch.empty(plan.yshape(), device=dev)
        call = lambda: tcprod.tc_cprod(plan.handle, src, dst)
    else:
        lowp_dt = torch.bfloat16 if args.precision in ("bf16", "bf16x3") else torch.float32
        planes = 3 if args.precision == "bf16x3" else 1
        roof_kernel = ("k_umma_gemm (tcgen05 slice GEMMs of one product"
                       + (", six split-BF16 products)" if planes == 3 else ")")
                       if args.precision != "fp32" else "k_slice_gemm (FFMA slice GEMMs of one product)")
        src = torch.randn((planes * n3, n2, s), device=dev).to(lowp_dt)
        dst = torch.empty((n3, n1, s), device=dev)
        call = lambda: tcprod.tc_slice_gemm(plan.handle, src, dst)
        reps = 50
    prod_ms = graph_time(call, reps)
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
    inf = tcprod.read_info(info)

    t_max, value = replica_throughput(total_ms, args.steps, iters, world, dev)
    if rank == 0:
        peaks, src_peaks = load_peaks()
        sm_max = peaks.get("sm_max_mhz", 2070.0)
        fp32_peak = FP32_LANES * 2 * sm_max * 1e6 / 1e12
        achieved = fl / (prod_ms * 1e-3) / 1e12
        if args.precision == "fp32":
            traffic = captured_traffic("k_cprod2") if roof_kernel.startswith("k_cprod2") and \
                args.workload == "two_sided_256" else None
            roof = {"kernel": roof_kernel, "bound": "alu", "achieved": achieved, "peak": fp32_peak,
                    "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic,
                    "peak_source": f"152 SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz "
                                   f"({src_peaks} max clock)", "launch_ms": prod_ms}
        elif args.precision == "bf16x3":  # six BF16 products per FP32-level product
            peak = peaks.get("bf16_tflops", FALLBACK_BF16_TFLOPS) / 6.0
            roof = {"kernel": roof_kernel, "bound": "tensor", "achieved": achieved, "peak": peak,
                    "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                    "peak_source": f"MEASURED_PEAKS.json bf16_tflops ({src_peaks}) / 6: each "
                                   "FP32-level product is six BF16 products",
                    "launch_ms": prod_ms, "algorithmic_flops": fl,
                    "note": "its 268 MB at the measured HBM rate take 40 us at 512x512x64, "
                            "less than the six products at the tensor rate"}
        else:  # tcgen05 GEMM: A~ and X~ in the input type read once, Y~ written in FP32
            es = {"bf16": 2, "bf16x3": 6}.get(args.precision, 4)
            gbytes = (n3 * n1 * n2 + n3 * n2 * s) * es + n3 * n1 * s * 4
            hbm = peaks.get("hbm_gbs", FALLBACK_HBM_GBS)
            gbs = gbytes / (prod_ms * 1e-3) / 1e9
            roof = {"kernel": roof_kernel, "bound": "hbm", "achieved": gbs, "peak": hbm,
                    "unit": "GB/s", "frac": gbs / hbm, "traffic": None,
                    "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({src_peaks})",
                    "launch_ms": prod_ms, "algorithmic_bytes": gbytes,
                    "note": ("the mode-3 transform passes take most of this solve; see profiles"
                             if args.product == "th" else
                             "transform-domain iteration: the solve runs the fused form of "
                             "this GEMM (Krylov epilogue and BF16 copy in the store, 235 MB a "
                             "product at 512x512x64); timed here is the plain form; see "
                             "profiles")}
        line = {
            "metric": METRIC, "value": value, "unit": "LSQR iterations/s",
            "solves_per_s": value / iters, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "bf16x3": "f32-level: three BF16 planes an operand, six products, f32 accumulate"}.get(args.precision, f"{args.precision} GEMM inputs, f32"),
            "data": "synthetic (seeded image + Gaussian blur + 1e-3 noise)",
            "config": {"workload": f"{args.workload}: c-LSQR {iters} it + Tikhonov/GCV, "
                                   f"A {n1}x{n2}x{n3}" + (f", B {s}x{s}x{n3}" if two else "")
                                   + f", X {n2}x{s}x{n3}",
                       "precision": args.precision, "product": args.product,
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roof,
            "e2e": {"value": iters / (e2e_ms / 1000.0) * world, "unit": "LSQR iterations/s",
                    "h2d_bytes_per_step": int(C.numel() * 4),
                    "d2h_bytes_per_step": int(Xr.numel() * 4 + info.numel())},
            "gpu_launches": args.steps * lsqr_kernel_launches(iters, two, n3 <= 4,
                                                              precision=args.precision, s=s,
                                                              n3=n3),
            "clocks": clk,
            "solve": {"iters": inf["iters"], "status": inf["status"], "lambda": inf["lam"],
                      "resid": inf["resid"],
                      "rel_err_reg": float((Xr - Xt).norm() / Xt.norm()),
                      "rel_err_lsqr": float((X - Xt).norm() / Xt.norm())},
        }
        if not args.no_precision_forms and world == 1:
            line["precision_forms"] = precision_forms(dev, peaks)
            line["batched_form"] = batched_form(dev)
            line["learned_form"] = learned_form()
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    cb_steps = []
    cores = len(os.sched_getaffinity(0))
    budget = 4.0  # seconds of oracle work per step (the worker warms up first)
    t0 = time.perf_counter()
    total_iters = 0
    for _ in range(args.steps):
        cb = cpu_baseline(args.workload, budget_s=budget)
        cb_steps.append(cb)
        total_iters += 1
    el = time.perf_counter() - t0
    value = statistics.median(c["value"] for c in cb_steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "LSQR iterations/s",
        "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": el * 1000.0 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded image + Gaussian blur)",
        "config": {"workload": f"{args.workload}: c-LSQR {wl['iters']} it (FP64 NumPy oracle "
                               "on the host cores; each step a bounded sample)"},
        "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value,
                         "unit": "LSQR iterations/s", "sample": cb_steps[0]["sample"]},
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
    ap.add_argument("--workload", default="two_sided_256", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision-forms", action="store_true")
    ap.add_argument("--iters", type=int, default=0, help="override the workload's iterations")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tf32", "bf16", "bf16x3"],
                    help="slice-GEMM inputs of the main workload (tensor-core forms need "
                         "one-sided plans: video_512 or colour_64)")
    ap.add_argument("--product", default="th", choices=["th", "orthodct"],
                    help="c-product reading: Definition 2.1 (th) or Algorithm 1's dct "
                         "(orthodct; off the fused route LSQR then runs in the transform domain)")
    ap.add_argument("--paper-shaped", action="store_true",
                    help="time the paper's three methods on the shapes of its Tables 1-4")
    ap.add_argument("--cpu-worker", default=None)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    args = ap.parse_args()
    if args.cpu_worker:
        cpu_worker(args.cpu_worker, args.cpu_budget)
        return
    if args.paper_shaped:
        for row in paper_shaped():
            print(json.dumps(row))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
