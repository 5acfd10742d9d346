"""Timing of the library on the paper-shaped workloads other than the main
benchmark (one JSON line per case, CUDA-event times of whole calls after
warm-up, inputs resident on the device):

  left_small  : left-looking RHQR (Algorithm 4), W 4096 x 32 float64 Gaussian,
                Gaussian sketch k = 128, float64 -- latency per factorisation
  srht_left   : left-looking RHQR, W = A diag(sigma) B 2^20 x 128 (sigma 1 ..
                1e-12), SRHT k = 512, float64 and float32
  srht_rec    : recRHQR + refinement on the same matrix and sketch, float64
                (2 passes) and float32 (3 passes)
  arnoldi     : RHQR-Arnoldi steps (Algorithm 7) with the 2-D convection-
                diffusion operator on a 1024 x 1024 grid (n = 2^20, Peclet 10),
                SRHT k = 400, 100 steps, float64 and float32 basis; the operator
                (torch, matrix-free) is timed with the step, as a user runs it
  rgs         : BLAS2-RGS (Algorithm 9) of the srht_left matrix, float64 and
                float32, SRHT k = 512 (Omega_full, no exact top block)
  gmres       : restarted RHQR-GMRES (Algorithm 8) on the same system, restart
                100, float64, up to --cycles cycles towards 1e-8 (time per cycle
                and the relative residual after each)

python -m paper_2405_10923_gb300.workloads_case [--cases left_small srht_left srht_block srht_trim srht_rec rgs arnoldi gmres] [--reps 3]

Accuracy is reported with the library's own sketch of the result in float64
(orth = max |eig(I - (Psi Q)^t Psi Q)|) and resid = ||W - QR||_F / ||W||_F
computed with torch."""

from __future__ import annotations

import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def _time(fn, reps):
    import torch

    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cases", nargs="+", default=["left_small", "srht_left", "srht_block", "srht_trim", "srht_rec", "rgs", "arnoldi", "gmres"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--cycles", type=int, default=5)
    a = ap.parse_args()

    import numpy as np
    import torch

    import paper_2405_10923_gb300 as rh
    import rhqr_inputs as ri
    from paper_2405_10923_gb300 import torch_api as ta

    rh.load()

    def metrics(sk, W, out, m):
        Q, R = out["Q"], out["R"]
        Z = sk.apply(rh.colmajor(Q.double()), m)
        G = (Z.t() @ Z).cpu().numpy()
        orth = float(np.max(np.abs(np.linalg.eigvalsh(np.eye(m) - G))))
        W64 = W.double()
        resid = float(torch.linalg.norm(W64 - Q.double() @ R) / torch.linalg.norm(W64))
        return orth, resid

    def emit(**kw):
        print(json.dumps(kw), flush=True)

    if "left_small" in a.cases:
        n, m, k = 4096, 32, 128
        W = rh.colmajor(torch.tensor(ri.gaussian(n, m, 1001), dtype=torch.float64, device="cuda"))
        sk = ta.Sketch(n, k, rh.GAUSSIAN, 2001, rh.F64)
        opts = ta.make_opts(alg=rh.ALG_LEFT)
        out = ta.factor(sk, W, opts=opts)
        ms = _time(lambda: ta.factor(sk, W, opts=opts, out=out, ws=out["ws"]), max(a.reps, 20))
        orth, resid = metrics(sk, W, out, m)
        emit(case="left_small", path="left-looking RHQR float64", n=n, m=m, k=k, sketch="gaussian f64",
             us_per_factorisation=ms * 1e3, orth=orth, resid=resid)
        sk.close()

    n, m, k = 1 << 20, 128, 512
    W64 = None
    if any(c in a.cases for c in ("srht_left", "srht_rec", "rgs", "srht_block", "srht_trim")):
        W64 = ri.device_spectrum(n, m, 1e12, 1002, dtype=torch.float64)
        W32 = ri.device_spectrum(n, m, 1e12, 1002, dtype=torch.float32)
        sk = ta.Sketch(n, k, rh.SRHT, 2002)
    if "srht_left" in a.cases:
        for W, name in ((W64, "f64"), (W32, "f32")):
            opts = ta.make_opts(alg=rh.ALG_LEFT)
            out = ta.factor(sk, W, opts=opts)
            ms = _time(lambda: ta.factor(sk, W, opts=opts, out=out, ws=out["ws"]), a.reps)
            orth, resid = metrics(sk, W, out, m)
            es = W.element_size()
            emit(case="srht_left", path="left-looking RHQR " + name, n=n, m=m, k=k, sketch="srht",
                 ms=ms, gbps_w_factored=n * m * es / (ms * 1e-3) / 1e9,
                 u_traffic_gb=n * (m * (m - 1) / 2 + 3 * m) * es / 1e9, orth=orth, resid=resid)
    if "srht_block" in a.cases:
        for W, name in ((W64, "f64"), (W32, "f32")):
            for bs in (16, 32, 64):
                opts = ta.make_opts(alg=rh.ALG_BLOCK, block_size=bs)
                out = ta.factor(sk, W, opts=opts)
                ms = _time(lambda: ta.factor(sk, W, opts=opts, out=out, ws=out["ws"]), a.reps)
                orth, resid = metrics(sk, W, out, m)
                es = W.element_size()
                emit(case="srht_block", path=f"blockRHQR {name}, blocks of {bs}", n=n, m=m, k=k, sketch="srht",
                     ms=ms, gbps_w_factored=n * m * es / (ms * 1e-3) / 1e9, orth=orth, resid=resid)
    if "srht_trim" in a.cases:
        for kt in (k, 96):  # the sketch size of the other cases, and fewer rows than columns
            skt = ta.Sketch(n, kt, rh.SRHT, 2002)
            for W, name in ((W64, "f64"), (W32, "f32")):
                out = ta.trim_factor(skt, W)
                ms = _time(lambda: ta.trim_factor(skt, W), a.reps)
                Q, R = out["Q"], out["R"]
                W64c = W.double()
                resid = float(torch.linalg.norm(W64c - Q.double() @ R) / torch.linalg.norm(W64c))
                sv = torch.linalg.svdvals(Q.double())
                emit(case="srht_trim", path=f"trimRHQR left-looking {name}", n=n, m=m, k=kt, sketch="srht", ms=ms,
                     gbps_w_factored=n * m * W.element_size() / (ms * 1e-3) / 1e9, resid=resid,
                     cond_q=float(sv[0] / sv[-1]), status=ta.read_info(out["info"])["status"])
            skt.close()
    if "srht_rec" in a.cases:
        for W, name, passes in ((W64, "f64", 2), (W32, "f32", 3)):
            opts = ta.make_opts(alg=rh.ALG_REC, passes=passes)
            out = ta.factor(sk, W, opts=opts)
            ms = _time(lambda: ta.factor(sk, W, opts=opts, out=out, ws=out["ws"]), a.reps)
            orth, resid = metrics(sk, W, out, m)
            es = W.element_size()
            emit(case="srht_rec", path=f"recRHQR {name}, {passes} passes", n=n, m=m, k=k, sketch="srht", ms=ms,
                 gbps_w_factored=n * m * es / (ms * 1e-3) / 1e9, orth=orth, resid=resid)
    if "rgs" in a.cases:
        for W, name in ((W64, "f64"), (W32, "f32")):
            ta.blas2_rgs(sk, W)
            ms = _time(lambda: ta.blas2_rgs(sk, W), a.reps)
            Q, R, T, S, info = ta.blas2_rgs(sk, W)
            torch.cuda.synchronize()
            G = (S.t() @ S).cpu().numpy()
            emit(case="rgs", path="BLAS2-RGS " + name, n=n, m=m, k=k, sketch="srht", ms=ms,
                 gbps_w_factored=n * m * W.element_size() / (ms * 1e-3) / 1e9, status=ta.read_info(info)["status"],
                 sketched_orth=float(np.max(np.abs(np.linalg.eigvalsh(np.eye(m) - G)))),
                 t_minus_identity=float((T - torch.eye(m, dtype=T.dtype, device=T.device)).abs().max()),
                 resid=float(torch.linalg.norm(W.double() - Q.double() @ R) / torch.linalg.norm(W.double())))
    if "arnoldi" in a.cases:
        g = 1024
        n, mmax, k = g * g, 100, 400
        sk = ta.Sketch(n, k, rh.SRHT, 2005)
        for dt, name in ((torch.float64, "f64"), (torch.float32, "f32")):
            for nrhs in (1, 32):
                op = ta.StencilOperator(g, nrhs=nrhs)
                rng = np.random.default_rng(1005)
                if nrhs == 1:
                    b = torch.tensor(rng.standard_normal(n), dtype=dt, device="cuda")
                else:
                    b = ta.block(n, nrhs, dt).copy_(torch.tensor(rng.standard_normal((n, nrhs)), dtype=dt))
                arn = ta.Arnoldi(sk, n, mmax, dtype=dt, nrhs=nrhs)

                def cycle():
                    _, q = arn.begin(b)
                    for _ in range(mmax):
                        _, q = arn.step(op(q))
                    return q

                ms = _time(cycle, a.reps)
                emit(case="arnoldi", path=f"RHQR-Arnoldi {name} basis, {nrhs} right-hand side(s) per launch", n=n,
                     steps=mmax, k=k, nrhs=nrhs, sketch="srht", ms_per_cycle=ms, us_per_step=ms * 1e3 / mmax,
                     us_per_step_per_rhs=ms * 1e3 / mmax / nrhs,
                     basis_gb=n * (mmax + 1) * b.element_size() * nrhs / 1e9)
                arn.close()
        sk.close()
    if "gmres" in a.cases:
        g = 1024
        n, restart, k, nrhs = g * g, 100, 400, 32
        sk = ta.Sketch(n, k, rh.SRHT, 2005)
        op = ta.StencilOperator(g, nrhs=nrhs)
        B = ta.block(n, nrhs, torch.float64).copy_(
            torch.tensor(np.random.default_rng(1005).standard_normal((n, nrhs))))
        for dt, name in ((torch.float32, "f32 basis, f64 iterate"), (torch.float64, "f64 basis")):
            solver = ta.GMRES(sk, n, restart, dtype=dt, nrhs=nrhs)
            solver.solve(op, B, tol=1e-8, max_cycles=1)  # warm-up
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record()
            X, hist = solver.solve(op, B, tol=1e-8, max_cycles=a.cycles)
            t1.record()
            torch.cuda.synchronize()
            cycles = len(hist) - 1
            emit(case="gmres", path=f"restarted RHQR-GMRES, {name}", n=n, restart=restart, k=k, nrhs=nrhs,
                 sketch="srht", cycles=cycles, converged=bool(hist[-1] <= 1e-8), total_s=t0.elapsed_time(t1) / 1e3,
                 ms_per_cycle=t0.elapsed_time(t1) / max(cycles, 1),
                 max_relative_residuals=[float(f"{h:.3e}") for h in hist])
            solver.close()
        sk.close()


if __name__ == "__main__":
    main()
