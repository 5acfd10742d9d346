"""One factorisation case for profiling (ncu) and quick timing.

python -m paper_2405_10923_gb300.profile_case --n 1048576 --m 256 --k 1024 \
    --alg rec --passes 1 --kind gaussian --sketch-dtype bf16 --reps 2

Builds W = A diag(sigma) B on the device (float32, cond 1e10 by default),
creates the sketch, runs rhqr_factor `reps` times and prints the phase times
of the last call (CUDA events of the library's profiler)."""

from __future__ import annotations

import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--m", type=int, default=256)
    ap.add_argument("--k", type=int, default=1024)
    ap.add_argument("--cond", type=float, default=1e10)
    ap.add_argument("--alg", choices=["rec", "left", "block"], default="rec")
    ap.add_argument("--block-size", type=int, default=32)
    ap.add_argument("--passes", type=int, default=1)
    ap.add_argument("--limbs", type=int, nargs=2, default=[2, 2])
    ap.add_argument("--kind", choices=["gaussian", "srht"], default="gaussian")
    ap.add_argument("--sketch-dtype", choices=["f64", "f32", "bf16", "f16"], default="bf16")
    ap.add_argument("--dtype", choices=["f32", "f64"], default="f32")
    ap.add_argument("--reps", type=int, default=2)
    a = ap.parse_args()

    import torch

    import paper_2405_10923_gb300 as rh
    import rhqr_inputs as ri
    from paper_2405_10923_gb300 import torch_api as ta

    rh.load()
    dt = torch.float32 if a.dtype == "f32" else torch.float64
    W = ri.device_spectrum(a.n, a.m, a.cond, 1003, dtype=dt)
    kind = rh.GAUSSIAN if a.kind == "gaussian" else rh.SRHT
    sdt = {"f64": rh.F64, "f32": rh.F32, "bf16": rh.BF16, "f16": rh.F16}[a.sketch_dtype]
    sk = ta.Sketch(a.n, a.k, kind, 2003, sdt)
    alg = {"rec": rh.ALG_REC, "left": rh.ALG_LEFT, "block": rh.ALG_BLOCK}[a.alg]
    opts = ta.make_opts(alg=alg, passes=a.passes, limbs_first=a.limbs[0], limbs_refine=a.limbs[1],
                        block_size=a.block_size)
    out = ta.factor(sk, W, opts=opts)
    for _ in range(a.reps - 1):
        rh.rhqr_profile_enable(True)
        ta.factor(sk, W, opts=opts, out=out, ws=out["ws"])
    torch.cuda.synchronize()
    phases = rh.rhqr_profile_read()
    rh.rhqr_profile_enable(False)
    print(json.dumps({"info": ta.info(out), "phases_ms": {k: v[0] for k, v in phases.items() if v[1]}}))


if __name__ == "__main__":
    main()
