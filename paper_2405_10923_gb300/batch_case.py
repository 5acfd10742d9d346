"""The batched workload for timing and profiling: many ragged tall-skinny
float32 problems, each with its own SRHT sketch (k_i = 4 m_i), factored by
rhqr_factor_batched and replayed as one CUDA graph.

python -m paper_2405_10923_gb300.batch_case --count 512 --n-lo 16384 --n-hi 262144 \
    --passes 3 --reps 5 [--tune-cache FILE] [--no-graph]

Prints one JSON line: the batch's size, the tuned launch shapes, the mean
graph-replay time (CUDA events; the batch's 11 GB of W and Q exceed L2), GB/s
of W factored, the phase times of one profiled (non-graph) run, the device
statuses, and for a few problems ||W - QR||_F / ||W||_F computed with torch."""

from __future__ import annotations

import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--n-lo", type=int, default=16384)
    ap.add_argument("--n-hi", type=int, default=262144)
    ap.add_argument("--m", type=int, nargs="+", default=[16, 32, 64, 128])
    ap.add_argument("--cond", type=float, default=1e8)
    ap.add_argument("--passes", type=int, default=3)
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--tune-cache", default=None)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    a = ap.parse_args()

    import torch

    import paper_2405_10923_gb300 as rh
    import rhqr_inputs as ri
    from paper_2405_10923_gb300 import torch_api as ta

    rh.load()
    dt = torch.float32 if a.dtype == "f32" else torch.float64
    Ws, ns, ms = ri.device_ragged_batch(a.count, a.n_lo, a.n_hi, a.m, a.cond, a.seed, dt)
    sks = [ta.Sketch(n, 4 * m, rh.SRHT, 7000 + i) for i, (n, m) in enumerate(zip(ns, ms))]
    b = ta.Batch(sks, Ws, passes=a.passes)
    choice = b.tuning() if a.no_tune else b.tune(reps=3, cache=a.tune_cache)

    rh.rhqr_profile_enable(True)
    l0 = rh.rhqr_launch_count()
    b.run()
    launches = rh.rhqr_launch_count() - l0
    torch.cuda.synchronize()
    phases = rh.rhqr_profile_read()
    rh.rhqr_profile_enable(False)

    st = torch.cuda.current_stream()
    g = None if a.no_graph else b.capture()
    launch = (lambda: g.replay()) if g is not None else (lambda: b.run())
    for _ in range(2):
        launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(a.reps):
        launch()
    e1.record(st)
    torch.cuda.synchronize()
    ms_per = e0.elapsed_time(e1) / a.reps
    es = 4 if a.dtype == "f32" else 8
    w_bytes = sum(n * m for n, m in zip(ns, ms)) * es

    infos = b.infos()
    bad = [i for i, x in enumerate(infos) if x["status"] != 0]
    resid = {}
    for i in sorted(set([0, 1, a.count // 2, a.count - 1])):
        W = Ws[i].double()
        QR = b.Q[i].double() @ b.R[i]
        resid[i] = float(torch.linalg.norm(W - QR) / torch.linalg.norm(W))
    print(json.dumps({
        "count": a.count, "rows": int(sum(ns)), "w_gb": w_bytes / 1e9, "passes": a.passes, "dtype": a.dtype,
        "tuning": {"a_threads": choice[0], "solve_rb": choice[1], "solve_cap": choice[2]},
        "graph": g is not None, "ms_per_batch": ms_per, "gbps_w_factored": w_bytes / ms_per / 1e6,
        "kernels_per_batch": launches,
        "phases_ms": {k: v[0] for k, v in phases.items() if v[1]},
        "failed": bad[:10], "residual_sampled": resid,
    }))
    b.close()


if __name__ == "__main__":
    main()
