#!/usr/bin/env python
"""Benchmark of the GB300 randomized Householder QR library.

Metric: GB/s of W factored by recRHQR (Algorithm 6 with refinement passes) on
W = A diag(sigma) B, n = 2^22 rows, m = 256 columns, float32, singular values
log-spaced from 1 to 1e-10, Gaussian sketch k = 1024 stored in bf16, sketch
products on tcgen05 tensor cores (float32 data split into bf16 limbs), small
Householder QR / T / R work in float64.  One step = one rhqr_factor call
(all passes) on device-resident data; W (4.3 GB) is larger than L2, so no
flush is needed.  Beside it: the plain FP64 GPU path on the same matrix, the
accuracy of both against the stated tolerances, an end-to-end number through
the library's host pipeline (every step copies W in from page-locked host memory
and Q, R back out; the copies of neighbouring steps overlap the factorisation),
and the FP64 CPU oracle timed on a bounded sample on the host cores.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Multi-GPU (torchrun): every rank factors its own matrix (independent
replicas, weak scaling); rank 0 prints the line with the max time over ranks.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GB/s of W factored (recRHQR n=2^22,m=256): mixed vs FP64 path at stated error"
UNIT = "GB/s"
SAMPLE_ROWS = 16384  # rows of the bounded CPU sample (same m, k, recipe)
REF_ROWS = 4096  # rows per step of the reference arm (about 4 s of CPU work each)

# DRAM bytes (read + write) per launch at n = 2^22, m = 256, k = 1024, from ncu
# captures at n = 2^20 scaled by 4 (both kernels stream W / Q and the operator in
# proportion to n); None when the kernel changed since the counters were taken.
TRAFFIC_BYTES = {"sketch": 4 * (3.2899e9 + 4.86e6), "solve": 4 * (1.0773e9 + 1.0140e9), "hqr": None}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=1 << 22)
    ap.add_argument("--m", type=int, default=256)
    ap.add_argument("--k", type=int, default=1024)
    ap.add_argument("--cond", type=float, default=1e10)
    ap.add_argument("--passes", type=int, default=3)
    ap.add_argument("--limbs", type=int, nargs=2, default=[2, 2])
    return ap.parse_args()


def workload(a):
    return {
        "workload": f"recRHQR mixed precision, W {a.n}x{a.m} float32 cond {a.cond:g}, Gaussian sketch k={a.k} "
                    f"(bf16 operator, tcgen05), {a.passes} passes",
        "n": a.n, "m": a.m, "k": a.k, "cond": a.cond, "passes": a.passes,
        "limbs_first_refine": list(a.limbs), "sketch_dtype": "bf16", "data_dtype": "f32",
        "small_side_dtype": "f64", "l2": "inputs larger than L2 (W is n*m*4 bytes), no flush",
    }


def cores_used() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample_run(a, seed: int, rows: int = SAMPLE_ROWS):
    """The FP64 oracle (as it stands) on a bounded sample: same m, k, recipe."""
    import numpy as np

    import rhqr_inputs as ri
    from oracle import rhqr, sketch

    ns = min(rows, a.n)
    W = ri.spectrum(ns, a.m, a.cond, seed).astype(np.float32).astype(np.float64)
    sk = sketch.GaussianSketch(ns, a.k, seed + 1, "bf16")
    t0 = time.perf_counter()
    rhqr.rec_rhqr_refined(W, sk, passes=a.passes)
    dt = time.perf_counter() - t0
    return ns, dt


def cpu_baseline(a, seed=77):
    ns, dt = oracle_sample_run(a, seed)
    return {
        "value": ns * a.m * 4 / dt / 1e9, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
        "sample": f"recRHQR {a.passes} passes on {ns} of the {a.n} rows (m={a.m}, k={a.k}, bf16 Gaussian "
                  f"operator values, float64 arithmetic, numpy/LAPACK); {dt:.1f} s",
    }


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_id: str):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, flag in zip(self.NAMES, parts[3:7]):
                if flag.lower() in ("active", "1", "0x1"):
                    reasons.add(name)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time, returned on every rank (unchanged on one process)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, bytes_per_rank: int, ms: float) -> float:
    """GB/s of W factored by `world` replicas that each factor bytes_per_rank in ms."""
    return world * bytes_per_rank / (ms * 1e-3) / 1e9


def measured_peaks():
    """HBM copy bandwidth and the burst bf16 rate: the dominant kernel is timed
    per launch (about 4 ms each, inside a step of under 30 ms), not as a
    seconds-long loop, so the burst figure is its denominator."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    except (OSError, ValueError):
        return 6800.0, 1900.0, "fallback"


# ---------------------------------------------------------------------------
# reference arm: the oracle
# ---------------------------------------------------------------------------


def run_reference(a, rank: int, world: int):
    if rank != 0:
        return
    for i in range(a.warmup):
        oracle_sample_run(a, 77 + i, REF_ROWS)
    times = []
    ns = 0
    for i in range(a.steps):
        ns, dt = oracle_sample_run(a, 177 + i, REF_ROWS)
        times.append(dt)
    t = sum(times) / len(times)
    v = ns * a.m * 4 / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload(a),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
                         "sample": f"recRHQR {a.passes} passes on {ns} of the {a.n} rows per step"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------


def run_ours(a, rank: int, world: int, local_rank: int):
    import numpy as np
    import torch

    import paper_2405_10923_gb300 as rh
    import rhqr_inputs as ri
    from paper_2405_10923_gb300 import torch_api as ta

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    rh.load()
    dist = None
    if world > 1:
        import torch.distributed as dist

    def barrier():
        if dist is not None:
            dist.barrier()

    n, m, k = a.n, a.m, a.k
    W = ri.device_spectrum(n, m, a.cond, 1003 + rank)
    sk = ta.Sketch(n, k, rh.GAUSSIAN, 2003 + rank, rh.BF16)
    opts = ta.make_opts(alg=rh.ALG_REC, passes=a.passes, limbs_first=a.limbs[0], limbs_refine=a.limbs[1])
    out = ta.factor(sk, W, opts=opts)
    ws = out["ws"]
    for _ in range(a.warmup):
        ta.factor(sk, W, opts=opts, out=out, ws=ws)
    torch.cuda.synchronize()
    info = ta.info(out)
    if info["status"] != 0:
        raise RuntimeError(f"factorisation failed: {info}")

    # ---- timed region: K steps on device-resident data
    props = torch.cuda.get_device_properties(dev)
    gpu_id = str(getattr(props, "uuid", local_rank))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) == 36:
        gpu_id = "GPU-" + gpu_id
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(gpu_id)
    time.sleep(0.3)
    rh.rhqr_profile_enable(True)
    l0 = rh.rhqr_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        ta.factor(sk, W, opts=opts, out=out, ws=ws)
    e1.record()
    torch.cuda.synchronize()
    launches = rh.rhqr_launch_count() - l0
    phases = rh.rhqr_profile_read()
    rh.rhqr_profile_enable(False)
    clk = clocks.stop()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / a.steps, dist, dev)
    bytes_w = n * m * 4
    value = replica_throughput(world, bytes_w, ms)

    # ---- accuracy of the mixed path (Psi Q accumulated in float64, same operator)
    def orth(skh, Q):
        Z = skh.apply(rh.colmajor(Q.double()), m)
        G = Z.t() @ Z
        return float(np.max(np.abs(np.linalg.eigvalsh(np.eye(m) - G.cpu().numpy()))))

    def resid(Wt, Q, R):
        W64 = Wt.double()
        return float(torch.linalg.norm(W64 - Q.double() @ R) / torch.linalg.norm(W64))

    acc_mixed = {"orth": orth(sk, out["Q"]), "resid": resid(W, out["Q"], out["R"]), "passes": a.passes,
                 "tolerance": 1e-5}

    # ---- end to end: every step copies W in from page-locked host memory and Q,
    #      R back out, through the library's host pipeline (the copies of step
    #      i+1 / i-1 overlap the factorisation of step i on separate streams)
    Wh = ta.Pipeline.host_colmajor(n, m, torch.float32)
    Wh.copy_(W)
    Qh = [ta.Pipeline.host_colmajor(n, m, torch.float32) for _ in range(2)]
    Rh = [ta.Pipeline.host_colmajor(m, m, torch.float64) for _ in range(2)]
    pipe = ta.Pipeline(sk, n, m, dtype=torch.float32, opts=opts, depth=2)
    pipe.submit(Wh, Qh[0], Rh[0])
    pipe.wait()
    # raw link bandwidth, for reading the end-to-end figure
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    W.t().copy_(Wh.t(), non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    h2d_gbs = bytes_w / (e0.elapsed_time(e1) * 1e-3) / 1e9
    e0.record()
    Qh[1].t().copy_(out["Q"].t(), non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    d2h_gbs = bytes_w / (e0.elapsed_time(e1) * 1e-3) / 1e9
    # both directions at once (W in on one stream, Q out on another): whether
    # this host link carries them concurrently decides whether the pipeline's
    # copy-in and copy-out can overlap each other
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    e0.record()
    s_in.wait_event(e0)
    s_out.wait_event(e0)
    with torch.cuda.stream(s_in):
        W.t().copy_(Wh.t(), non_blocking=True)
    with torch.cuda.stream(s_out):
        Qh[1].t().copy_(out["Q"].t(), non_blocking=True)
    torch.cuda.current_stream().wait_stream(s_in)
    torch.cuda.current_stream().wait_stream(s_out)
    e1.record()
    torch.cuda.synchronize()
    both_gbs = 2.0 * bytes_w / (e0.elapsed_time(e1) * 1e-3) / 1e9
    e2e_steps = max(2, a.steps)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        pipe.submit(Wh, Qh[i % 2], Rh[i % 2])
    pipe.wait()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / e2e_steps, dist, dev)
    e2e_ok = bool(torch.equal(Qh[(e2e_steps - 1) % 2], out["Q"].cpu()))
    pipe.close()
    del Wh, Qh, pipe

    # ---- roofline of the dominant phase (live CUDA events on the launching stream)
    hbm, bf16_peak, peak_src = measured_peaks()
    dom = max(("sketch", "solve", "hqr"), key=lambda p: phases[p][0])
    dom_ms = phases[dom][0] / max(1, phases[dom][1])
    if dom == "sketch":
        flops = 2.0 * k * (n - m) * m
        achieved = flops / (dom_ms * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
                "frac": achieved / bf16_peak, "peak_source": f"{peak_src} bf16 burst",
                "work": "algorithmic 2 k (n - m) m flop per launch (one bf16 product; the kernel issues one per "
                        "limb of X)"}
    elif dom == "solve":
        byts = 2.0 * n * m * 4
        achieved = byts / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_source": f"{peak_src} copy bandwidth"}
    else:
        p_rows = k + m
        flops = 2.0 * p_rows * m * m - 2.0 * m ** 3 / 3.0  # Householder QR of the (k+m) x m sketch
        peak = 1250.0  # GFLOP/s: nominal GB300 FP64 rate
        achieved = flops / (dom_ms * 1e-3) / 1e9
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GFLOP/s", "frac": achieved / peak,
                "peak_source": "nominal FP64 rate (1.25 TFLOP/s)"}
    roof["kernel"] = dom
    roof["ms_per_launch"] = dom_ms
    roof["traffic"] = TRAFFIC_BYTES.get(dom)
    phase_ms = {p: {"ms_per_step": v[0] / a.steps, "calls": v[1]} for p, v in phases.items() if v[1]}

    # ---- the same workload with the operator stored in fp16 (the other 16-bit
    #      format of the tensor-core sketch), same passes and limbs
    sk16 = ta.Sketch(n, k, rh.GAUSSIAN, 2003 + rank, rh.F16)
    out16 = ta.factor(sk16, W, opts=opts, out=out, ws=ws)
    for _ in range(a.warmup):
        ta.factor(sk16, W, opts=opts, out=out, ws=ws)
    torch.cuda.synchronize()
    h0e, h1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0e.record()
    for _ in range(a.steps):
        ta.factor(sk16, W, opts=opts, out=out, ws=ws)
    h1e.record()
    torch.cuda.synchronize()
    ms16 = h0e.elapsed_time(h1e) / a.steps
    fp16 = {"value": bytes_w / (ms16 * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms16, "steps": a.steps,
            "orth": orth(sk16, out16["Q"]), "resid": resid(W, out16["Q"], out16["R"]), "tolerance": 1e-5,
            "status": ta.info(out16)["status"]}
    sk16.close()

    # ---- the plain FP64 GPU path on the same matrix (2 passes), median of 5
    W64 = rh.colmajor(W.double())
    del out, ws, out16
    torch.cuda.empty_cache()
    sk64 = ta.Sketch(n, k, rh.GAUSSIAN, 2003 + rank, rh.F64)
    o64 = ta.make_opts(alg=rh.ALG_REC, passes=2)
    out64 = ta.factor(sk64, W64, opts=o64)
    torch.cuda.synchronize()
    runs64 = []
    for _ in range(5):
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record()
        ta.factor(sk64, W64, opts=o64, out=out64, ws=out64["ws"])
        f1.record()
        torch.cuda.synchronize()
        runs64.append(f0.elapsed_time(f1))
    ms64 = statistics.median(runs64)
    fp64 = {"value": bytes_w / (ms64 * 1e-3) / 1e9, "unit": UNIT, "ms": ms64, "ms_runs": runs64, "passes": 2,
            "orth": orth(sk64, out64["Q"]), "resid": resid(W64, out64["Q"], out64["R"]), "tolerance": 1e-12,
            "bytes_counted": "float32 bytes of W (same workload unit as the mixed path)"}
    sk64.close()

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16+f32+f64", "data": "synthetic",
        "config": dict(workload(a), parallelism=("replicas" if world > 1 else "single")),
        "accuracy": acc_mixed, "fp16_operator": fp16, "fp64_path": fp64,
        "speedup_vs_fp64_path": value / world / fp64["value"],
        "roofline": roof, "phases": phase_ms,
        "cpu_baseline": cpu_baseline(a),
        "e2e": {"value": replica_throughput(world, bytes_w, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": bytes_w,
                "d2h_bytes_per_step": bytes_w + m * m * 8, "steps": e2e_steps, "ms_per_step": e2e_ms,
                "path": "rhqr_pipeline (host W in, host Q and R out; copies overlap neighbouring steps)",
                "link_h2d_gbs": h2d_gbs, "link_d2h_gbs": d2h_gbs, "link_both_directions_gbs": both_gbs,
                "q_equals_device_path": e2e_ok},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def main():
    a = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_ours(a, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
