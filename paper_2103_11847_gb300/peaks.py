"""Measured peak rates of the GPU this runs on, for the roofline fractions:
FP32 FFMA, FP64 DFMA, tcgen05 TF32 and BF16 MMA issue rates (tc_peak_probe,
the library's own probe kernels), and, for reference, cuBLAS's FP32, TF32 and
FP64 GEMM rates through torch.matmul. Each rate is the best of several CUDA
event-timed launches; SM clocks are sampled with nvidia-smi meanwhile.

  python -m paper_2103_11847_gb300.peaks [out.json]

writes profiles/peaks.json by default.
"""
import json
import os
import subprocess
import sys
import time

import torch

from . import tcprod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _time(call, reps=5):
    """Best CUDA-event time (ms) of `call` over `reps` runs after a warm-up."""
    st = torch.cuda.current_stream()
    call()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        call()
        e1.record(st)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def probe_rates():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    status = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = {}
    # FFMA / DFMA: 8 CTAs x 256 threads a SM, 8 FMAs a thread and iteration
    threads = sms * 8 * 256
    for key, kind, iters in (("fp32_ffma_tflops", 0, 20000), ("fp64_dfma_tflops", 1, 2000)):
        ms = _time(lambda: tcprod.tc_peak_probe(kind, iters, status))
        out[key] = 2.0 * 8 * iters * threads / (ms * 1e-3) / 1e12
        out[key + "_ms"] = ms
    # tcgen05: four 128 x 256 x K MMAs an iteration on every SM
    for key, kind, iters, k in (("tf32_mma_tflops", 2, 4000, 8), ("bf16_mma_tflops", 3, 4000, 16)):
        ms = _time(lambda: tcprod.tc_peak_probe(kind, iters, status))
        out[key] = 2.0 * 128 * 256 * k * 4 * iters * sms / (ms * 1e-3) / 1e12
        out[key + "_ms"] = ms
    torch.cuda.synchronize()
    out["probe_status"] = int(status[0].item())
    return out


def cublas_rates(n=8192):
    out = {}
    prev = torch.backends.cuda.matmul.allow_tf32
    for key, dt, tf32 in (("cublas_sgemm_tflops", torch.float32, False),
                          ("cublas_tf32_tflops", torch.float32, True),
                          ("cublas_dgemm_tflops", torch.float64, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        m = n if dt != torch.float64 else n // 2
        a = torch.randn(m, m, device="cuda", dtype=dt)
        b = torch.randn(m, m, device="cuda", dtype=dt)
        ms = _time(lambda: torch.matmul(a, b), reps=3)
        out[key] = 2.0 * m ** 3 / (ms * 1e-3) / 1e12
        del a, b
    torch.backends.cuda.matmul.allow_tf32 = prev
    return out


def sample_clocks(seconds_fn):
    """Run seconds_fn() while nvidia-smi samples the SM clock every 100 ms."""
    q = "clocks.sm,clocks.max.sm,clocks_event_reasons.active"
    try:
        proc = subprocess.Popen(["nvidia-smi", "-i", "0", f"--query-gpu={q}",
                                 "--format=csv,noheader,nounits", "-lms", "100"],
                                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return seconds_fn(), None
    time.sleep(0.3)
    res = seconds_fn()
    proc.terminate()
    rows = []
    try:
        outs, _ = proc.communicate(timeout=5)
        for line in outs.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 2 and parts[0].replace(".", "").isdigit():
                rows.append((float(parts[0]), float(parts[1]), parts[2] if len(parts) > 2 else ""))
    except subprocess.TimeoutExpired:
        proc.kill()
    sm = sorted(r[0] for r in rows)
    clocks = {"samples": len(rows), "sm_mhz_median": sm[len(sm) // 2] if sm else None,
              "sm_max_mhz": max((r[1] for r in rows), default=None)}
    return res, clocks


def main(path=None):
    path = path or os.path.join(ROOT, "profiles", "peaks.json")
    torch.cuda.set_device(0)
    tcprod.lib()
    rates, clocks = sample_clocks(lambda: {**probe_rates(), **cublas_rates()})
    rec = {"gpu": torch.cuda.get_device_name(0), "sms":
           torch.cuda.get_device_properties(0).multi_processor_count, **rates,
           "clocks": clocks,
           "how": "tc_peak_probe kernels (FFMA/DFMA: 8 independent chains a thread, 8 CTAs "
                  "x 256 threads a SM; tcgen05: one CTA a SM issuing 128x256xK MMAs into "
                  "tensor memory) and torch.matmul (cuBLAS) on 8192^2 FP32/TF32 and 4096^2 "
                  "FP64; best of 5 (3) CUDA-event-timed runs after a warm-up",
           "command": "python -m paper_2103_11847_gb300.peaks"}
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))
    if rates.get("probe_status", 0) != 0:
        sys.exit(1)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else None)
