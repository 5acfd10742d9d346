"""Torch-tensor conveniences over the C ABI: they allocate outputs and the
workspace with torch and call the entry points of ``include/rhqr.h``.  No
arithmetic of the method happens here."""

from __future__ import annotations

import json
import os

import torch

from . import (ALG_LEFT, ALG_REC, BF16, F16, F32, F64, GAUSSIAN, SRHT, colmajor, dtype_code, ld_of, read_info,
               rhqr_batch_create, rhqr_batch_destroy, rhqr_batch_get_tuning, rhqr_batch_set_tuning, rhqr_batch_tune,
               rhqr_batch_workspace_size, rhqr_factor_batched, rhqr_arnoldi_begin, rhqr_arnoldi_create_batch,
               rhqr_stencil_apply, rhqr_stencil_residual, rhqr_stencil_residual_workspace, rhqr_arnoldi_solution_x, rhqr_arnoldi_destroy, rhqr_arnoldi_export, rhqr_arnoldi_step,
               rhqr_default_opts, rhqr_factor, rhqr_pipeline_create, rhqr_pipeline_destroy, rhqr_pipeline_submit,
               rhqr_pipeline_wait, rhqr_arnoldi_solution, rhqr_blas2_rgs, rhqr_blas2_rgs_workspace, rhqr_reconstruct,
               rhqr_trim_factor, rhqr_trim_workspace, rhqr_sketch_apply_rows,
               rhqr_sketch_apply_rows_workspace, rhqr_sketch_apply, rhqr_sketch_apply_workspace,
               rhqr_sketch_create, rhqr_sketch_destroy, rhqr_sketch_export, rhqr_sketch_shape, rhqr_workspace_size)

TORCH_DTYPE = {F64: torch.float64, F32: torch.float32, BF16: torch.bfloat16, F16: torch.float16}
__all__ = ["Sketch", "Arnoldi", "GMRES", "StencilOperator", "block", "Batch", "Pipeline", "factor", "trim_factor", "reconstruct", "colmajor", "ALG_LEFT", "ALG_REC", "GAUSSIAN", "SRHT"]


class Sketch:
    """Owner of an rhqr_sketch handle."""

    def __init__(self, n: int, k: int, kind: int, seed: int, omega_dtype: int = F64, stream=None):
        self.handle = rhqr_sketch_create(n, k, kind, seed, omega_dtype, stream)
        self.n, self.k, self.kind, self.N, self.omega_dtype = rhqr_sketch_shape(self.handle)

    def close(self):
        if self.handle:
            rhqr_sketch_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def export(self, device="cuda"):
        if self.kind == SRHT:
            signs = torch.empty(self.N, dtype=torch.int8, device=device)
            rows = torch.empty(self.k, dtype=torch.int32, device=device)
            rhqr_sketch_export(self.handle, signs, rows, None, 0)
            return {"signs": signs, "rows": rows}
        G = torch.empty((self.k, self.n), dtype=TORCH_DTYPE[self.omega_dtype], device=device)
        rhqr_sketch_export(self.handle, None, None, G, self.n)
        return {"G": G}

    def apply_rows(self, X_local: torch.Tensor, m: int, row0: int) -> torch.Tensor:
        """One row shard's share Psi_m[:, row0:row0+rows] X_local of the sketch
        (rhqr_sketch_apply_rows); the shards' results sum to apply(X, m)."""
        rows, c = X_local.shape
        ws_b = rhqr_sketch_apply_rows_workspace(self.handle, m, dtype_code(X_local), row0, rows, c)
        ws = torch.empty(max(ws_b, 1), dtype=torch.uint8, device=X_local.device)
        Z = colmajor(torch.zeros((self.k + m, c), dtype=torch.float64, device=X_local.device))
        rhqr_sketch_apply_rows(self.handle, m, X_local, dtype_code(X_local), row0, rows, c, ld_of(X_local), Z, ld_of(Z),
                               ws, ws_b)
        return Z

    def apply(self, X: torch.Tensor, m: int) -> torch.Tensor:
        """Z = Psi_m X (Algorithm 1), X column-major n x c."""
        n, c = X.shape
        ws_b = rhqr_sketch_apply_workspace(self.handle, m, dtype_code(X), n, c)
        ws = torch.empty(max(ws_b, 1), dtype=torch.uint8, device=X.device)
        Z = colmajor(torch.zeros((self.k + m, c), dtype=torch.float64, device=X.device))
        rhqr_sketch_apply(self.handle, m, X, dtype_code(X), n, c, ld_of(X), Z, ld_of(Z), ws, ws_b)
        return Z


def make_opts(alg=ALG_REC, passes=1, limbs_first=2, limbs_refine=2, want_U=False, want_Q=True, scaling=0,
              wait_budget=0, solve=0, block_size=32, column_scaling=0):
    o = rhqr_default_opts()
    o.alg, o.passes, o.limbs_first, o.limbs_refine = alg, passes, limbs_first, limbs_refine
    o.want_U, o.want_Q, o.scaling, o.wait_budget, o.solve = int(want_U), int(want_Q), scaling, wait_budget, solve
    o.block_size, o.column_scaling = block_size, int(column_scaling)
    return o


class Workspace:
    """A reusable device workspace for rhqr_factor."""

    def __init__(self, nbytes: int, device="cuda"):
        self.nbytes = nbytes
        self.buf = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)


def factor_outputs(sk: Sketch, n: int, m: int, dtype: torch.dtype, want_U: bool, want_Q: bool, device="cuda"):
    p = sk.k + m
    return {
        "U": colmajor(torch.zeros((n, m), dtype=dtype, device=device)) if want_U else None,
        "S": colmajor(torch.zeros((p, m), dtype=torch.float64, device=device)),
        "T": colmajor(torch.zeros((m, m), dtype=torch.float64, device=device)),
        "R": colmajor(torch.zeros((m, m), dtype=torch.float64, device=device)),
        "Q": colmajor(torch.zeros((n, m), dtype=dtype, device=device)) if want_Q else None,
        "info": torch.zeros(4, dtype=torch.int32, device=device),
    }


def factor(sk: Sketch, W: torch.Tensor, opts=None, out=None, ws: Workspace | None = None, stream=None, **kw):
    """rhqr_factor on a column-major W; returns the dict of output tensors."""
    n, m = W.shape
    opts = opts or make_opts(**kw)
    wt = dtype_code(W)
    want_U = bool(opts.want_U) or opts.alg != ALG_REC
    if out is None:
        out = factor_outputs(sk, n, m, W.dtype, want_U, bool(opts.want_Q), W.device)
    need = rhqr_workspace_size(sk.handle, n, m, wt, opts)
    if ws is None or ws.nbytes < need:
        ws = Workspace(need, W.device)
    U, Q = out["U"], out["Q"]
    rhqr_factor(sk.handle, W, wt, n, m, ld_of(W), opts, U, ld_of(U) if U is not None else n, out["S"],
                ld_of(out["S"]), out["T"], out["R"], Q, ld_of(Q) if Q is not None else n, ws.buf, ws.nbytes,
                out["info"], stream)
    out["ws"] = ws
    return out


class Pipeline:
    """Owner of an rhqr_pipeline handle: host W in, host Q and R out, the
    transfers of consecutive submissions overlapped with the factorisations."""

    def __init__(self, sk: Sketch, n: int, m: int, dtype=torch.float32, opts=None, depth: int = 2):
        self.sk, self.n, self.m, self.dtype = sk, n, m, dtype
        self.handle = rhqr_pipeline_create(sk.handle, dtype_code(torch.empty(0, dtype=dtype)), n, m, opts, depth)

    @staticmethod
    def host_colmajor(rows: int, cols: int, dtype, pin: bool = True) -> torch.Tensor:
        """A page-locked host tensor of shape (rows, cols) in column-major order."""
        return torch.empty((cols, rows), dtype=dtype, pin_memory=pin).t()

    def submit(self, W: torch.Tensor, Q: torch.Tensor, R: torch.Tensor, S=None, T=None, info=None):
        """Enqueue one factorisation; W, Q (column-major, n x m), R (m x m, read
        as column-major) and the optional S, T, info are host tensors."""
        for t in (W, Q, R, S, T, info):
            if t is not None and t.device.type != "cpu":
                raise ValueError("pipeline buffers are host tensors")
        rhqr_pipeline_submit(self.handle, W, ld_of(W), Q, ld_of(Q), R, S, ld_of(S) if S is not None else 0, T, info)

    def wait(self):
        rhqr_pipeline_wait(self.handle)

    def close(self):
        if self.handle:
            rhqr_pipeline_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def blas2_rgs(sk: Sketch, W: torch.Tensor):
    """rhqr_blas2_rgs (Algorithm 9) on a column-major W; returns Q, R, T, S and info."""
    n, m = W.shape
    wt = dtype_code(W)
    Q = colmajor(torch.zeros((n, m), dtype=W.dtype, device=W.device))
    R = colmajor(torch.zeros((m, m), dtype=torch.float64, device=W.device))
    T = colmajor(torch.zeros((m, m), dtype=torch.float64, device=W.device))
    S = colmajor(torch.zeros((sk.k, m), dtype=torch.float64, device=W.device))
    info = torch.zeros(4, dtype=torch.int32, device=W.device)
    need = rhqr_blas2_rgs_workspace(sk.handle, wt, n, m)
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device=W.device)
    rhqr_blas2_rgs(sk.handle, W, wt, n, m, ld_of(W), Q, ld_of(Q), R, T, S, ws, need, info)
    return Q, R, T, S, info


def trim_factor(sk: Sketch, W: torch.Tensor, scaling: int = 0, want_Q: bool = True):
    """rhqr_trim_factor (left-looking trimRHQR, Section 7) on a column-major W;
    returns a dict with U, S (k x m), T, Tt, R, Q (or None) and info."""
    n, m = W.shape
    wt = dtype_code(W)
    dev = W.device
    out = {
        "U": colmajor(torch.zeros((n, m), dtype=W.dtype, device=dev)),
        "S": colmajor(torch.zeros((sk.k, m), dtype=torch.float64, device=dev)),
        "T": colmajor(torch.zeros((m, m), dtype=torch.float64, device=dev)),
        "Tt": colmajor(torch.zeros((m, m), dtype=torch.float64, device=dev)),
        "R": colmajor(torch.zeros((m, m), dtype=torch.float64, device=dev)),
        "Q": colmajor(torch.zeros((n, m), dtype=W.dtype, device=dev)) if want_Q else None,
        "info": torch.zeros(4, dtype=torch.int32, device=dev),
    }
    need = rhqr_trim_workspace(sk.handle, wt, n, m)
    ws = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    Q = out["Q"]
    rhqr_trim_factor(sk.handle, W, wt, n, m, ld_of(W), scaling, out["U"], ld_of(out["U"]), out["S"], ld_of(out["S"]),
                     out["T"], out["Tt"], out["R"], Q, ld_of(Q) if Q is not None else n, ws, need, out["info"])
    out["ws"] = ws
    return out


def reconstruct(sk: Sketch, S, T, R, Z, W, want_Q=True):
    n, m = W.shape
    U = colmajor(torch.zeros((n, m), dtype=W.dtype, device=W.device))
    Q = colmajor(torch.zeros((n, m), dtype=W.dtype, device=W.device)) if want_Q else None
    need = rhqr_workspace_size(sk.handle, n, m, dtype_code(W), None)
    ws = torch.empty(need, dtype=torch.uint8, device=W.device)
    rhqr_reconstruct(sk.handle, S, ld_of(S), T, R, Z, ld_of(Z), W, dtype_code(W), n, m, ld_of(W), U, ld_of(U), Q,
                     ld_of(Q) if Q is not None else n, ws, need)
    return U, Q


def info(out) -> dict:
    return read_info(out["info"])


class Arnoldi:
    """Owner of an rhqr_arnoldi handle (Algorithm 7 with a caller-applied
    operator) over nrhs processes at once.  Vectors are tensors of shape (n,)
    for one process or column-major (n, nrhs) blocks (see :func:`block`);
    the Hessenberg columns come back as (M,) or (M, nrhs)."""

    def __init__(self, sk: Sketch, n: int, mmax: int, dtype=torch.float64, scaling: int = 0, device="cuda",
                 nrhs: int = 1):
        self.n, self.mmax, self.M, self.dtype, self.device, self.nrhs = n, mmax, mmax + 1, dtype, device, nrhs
        self.k = sk.k
        self.handle = rhqr_arnoldi_create_batch(sk.handle, n, mmax, nrhs, dtype_code(torch.empty(0, dtype=dtype)),
                                                scaling)
        self.info = torch.zeros((nrhs, 4), dtype=torch.int32, device=device)

    def close(self):
        if self.handle:
            rhqr_arnoldi_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _vec(self, rows, dtype):
        if self.nrhs == 1:
            return torch.zeros(rows, dtype=dtype, device=self.device)
        return block(rows, self.nrhs, dtype, self.device)

    def begin(self, r0: torch.Tensor):
        h0 = self._vec(self.M, torch.float64)
        q = self._vec(self.n, self.dtype)
        rhqr_arnoldi_begin(self.handle, r0, h0, q, self.info)
        return h0, q

    def step(self, w: torch.Tensor):
        h = self._vec(self.M, torch.float64)
        q = self._vec(self.n, self.dtype)
        rhqr_arnoldi_step(self.handle, w, h, q, self.info)
        return h, q

    def solution(self, H: torch.Tensor, m: int, h0: torch.Tensor, x0=None, x=None):
        """rhqr_arnoldi_solution: y = argmin ||h0 - H[:m+1, :m] y|| and, when x0
        is given, x = x0 + Q_m y (into x, default a new tensor).  For one
        process H is the column-major (mmax+1) x mmax float64 matrix of the
        step outputs; for a batch, a (nrhs, mmax, mmax+1) tensor whose slice b
        holds process b's matrix column by column (see :meth:`hessenberg`)."""
        ldh = ld_of(H) if H.dim() == 2 else H.shape[2]
        y = self._vec(max(self.mmax, 1), torch.float64)
        res = torch.zeros(self.nrhs, dtype=torch.float64, device=self.device)
        if x0 is not None and x is None:
            x = torch.empty_like(x0)
        xdt = dtype_code(x0) if x0 is not None else dtype_code(torch.empty(0, dtype=self.dtype))
        rhqr_arnoldi_solution_x(self.handle, H, ldh, m, h0, x0, x, xdt, y, res)
        return y[:m], (res if self.nrhs > 1 else res[:1]), x

    def hessenberg(self):
        """Storage for the Hessenberg columns of all processes."""
        if self.nrhs == 1:
            return colmajor(torch.zeros((self.M, self.mmax), dtype=torch.float64, device=self.device))
        return torch.zeros((self.nrhs, self.mmax, self.M), dtype=torch.float64, device=self.device)

    def export(self):
        """U, S, T of every process (process b: U[:, b M:(b+1) M] ...); for one
        process as before."""
        B = self.nrhs
        U = colmajor(torch.zeros((self.n, self.M * B), dtype=self.dtype, device=self.device))
        S = colmajor(torch.zeros((self.k + self.M, self.M * B), dtype=torch.float64, device=self.device))
        T = torch.zeros((B, self.M, self.M), dtype=torch.float64, device=self.device)
        cnt = rhqr_arnoldi_export(self.handle, U, ld_of(U), S, ld_of(S), T)
        Tt = T.transpose(1, 2)
        return U, S, (Tt[0] if B == 1 else Tt), cnt


def block(rows: int, cols: int, dtype, device="cuda") -> torch.Tensor:
    """A zero column-major (rows, cols) tensor with leading dimension rows."""
    return torch.zeros((cols, rows), dtype=dtype, device=device).t()


class StencilOperator:
    """The library's matrix-free convection-diffusion operator on a g x g grid
    (rhqr_stencil_apply) and its restart residual (rhqr_stencil_residual)."""

    def __init__(self, g: int, peclet: float = 10.0, nrhs: int = 1, device="cuda"):
        self.g, self.pe, self.nrhs, self.n = g, peclet, nrhs, g * g
        self.wbytes = rhqr_stencil_residual_workspace(g, nrhs)
        self.work = torch.empty(max(self.wbytes, 1), dtype=torch.uint8, device=device)
        self.norms = torch.zeros(2 * nrhs, dtype=torch.float64, device=device)

    def __call__(self, X: torch.Tensor) -> torch.Tensor:
        Y = torch.empty_like(X) if X.dim() == 1 else block(self.n, X.shape[1], X.dtype, X.device)
        rhqr_stencil_apply(self.g, self.pe, X, dtype_code(X), 1 if X.dim() == 1 else X.shape[1], Y)
        return Y

    def residual(self, B: torch.Tensor, X: torch.Tensor, rdtype=None):
        """R = B - A X (formed in float64, returned in rdtype, default B's) and
        the device tensors ||B[:, b] - A X[:, b]||, ||B[:, b]||."""
        nr = 1 if B.dim() == 1 else B.shape[1]
        rdtype = rdtype or B.dtype
        R = torch.empty(B.shape, dtype=rdtype, device=B.device) if B.dim() == 1 else block(self.n, nr, rdtype, B.device)
        rhqr_stencil_residual(self.g, self.pe, B, X, dtype_code(B), nr, R, dtype_code(R), self.norms, self.work,
                              self.wbytes)
        return R, self.norms[0:2 * nr:2], self.norms[1:2 * nr:2]


class GMRES:
    """Restarted RHQR-GMRES (Algorithm 8) for nrhs right-hand sides at once,
    over the library's batched Arnoldi steps with a caller-applied operator A
    (a function of an (n,) vector or an (n, nrhs) column-major block).  Each
    cycle starts from R = B - A X (the library's residual kernel when A has a
    `residual` method, as StencilOperator does), takes up to `restart` steps,
    checks the sketched residuals ||h0 - H y|| (= ||Psi (b - A x)||) every
    `check` steps and updates every X by rhqr_arnoldi_solution; it stops when
    ||b - A x|| <= tol ||b|| for every right-hand side.  B and X may be wider
    than the basis dtype (float64 with a float32 basis): the residual is then
    formed in float64 and every cycle's float32 correction is added to the
    float64 iterate by the library (rhqr_arnoldi_solution_x)."""

    def __init__(self, sk: Sketch, n: int, restart: int, dtype=torch.float64, device="cuda", nrhs: int = 1):
        self.arn = Arnoldi(sk, n, restart, dtype=dtype, device=device, nrhs=nrhs)
        self.restart, self.n, self.dtype, self.device, self.nrhs = restart, n, dtype, device, nrhs
        self.H = self.arn.hessenberg()

    def close(self):
        self.arn.close()

    def _residual(self, A, B, X):
        """R = B - A X in the basis dtype, with the norms of the residual and of B."""
        if hasattr(A, "residual"):
            R, rn, bn = A.residual(B, X, rdtype=self.dtype)
            return R, rn.cpu().numpy(), bn.cpu().numpy()
        # a caller-supplied operator: its residual is the caller's arithmetic
        R = B - A(X)
        Rd, Bd = R.double(), B.double()
        if R.dim() == 1:
            return (R.to(self.dtype), torch.linalg.norm(Rd).reshape(1).cpu().numpy(),
                    torch.linalg.norm(Bd).reshape(1).cpu().numpy())
        return (R.to(self.dtype), torch.linalg.norm(Rd, dim=0).cpu().numpy(),
                torch.linalg.norm(Bd, dim=0).cpu().numpy())

    def solve(self, A, B: torch.Tensor, x0=None, tol: float = 1e-8, max_cycles: int = 50, check: int = 10):
        """Returns X and the history of max_b ||b - A x|| / ||b|| per cycle."""
        if x0 is not None:
            X = x0.clone() if B.dim() == 1 else block(self.n, B.shape[1], B.dtype, B.device).copy_(x0)
        else:
            X = torch.zeros_like(B) if B.dim() == 1 else block(self.n, B.shape[1], B.dtype, B.device)
        history = []
        for cycle in range(max_cycles):
            R, rn, bn = self._residual(A, B, X)
            rel = rn / bn
            history.append(float(rel.max()))
            if (rn <= tol * bn).all():
                return X, history
            h0, q = self.arn.begin(R)
            steps = 0
            for j in range(self.restart):
                h, q = self.arn.step(A(q))
                if self.nrhs == 1:
                    self.H[:, j] = h
                else:
                    self.H[:, j, :] = h.t()
                steps = j + 1
                if steps % check == 0 and steps < self.restart:
                    _, res, _ = self.arn.solution(self.H, steps, h0)
                    if (res.cpu().numpy() <= 0.5 * tol * bn).all():
                        break
            _, _, X = self.arn.solution(self.H, steps, h0, x0=X, x=X)
        _, rn, bn = self._residual(A, B, X)
        history.append(float((rn / bn).max()))
        return X, history


class Batch:
    """Owner of an rhqr_batch plan over ragged problems (W_i column-major,
    one SRHT Sketch each) and of its outputs Q_i, S_i, T_i, R_i, the per-problem
    info records and the workspace."""

    def __init__(self, sketches, Ws, opts=None, **kw):
        self.sketches = list(sketches)
        self.W = list(Ws)
        self.opts = opts or make_opts(**kw)
        dev = self.W[0].device
        wt = dtype_code(self.W[0])
        self.Q = [colmajor(torch.zeros(w.shape, dtype=w.dtype, device=dev)) for w in self.W]
        self.S = [colmajor(torch.zeros((sk.k + w.shape[1], w.shape[1]), dtype=torch.float64, device=dev))
                  for sk, w in zip(self.sketches, self.W)]
        self.T = [colmajor(torch.zeros((w.shape[1], w.shape[1]), dtype=torch.float64, device=dev)) for w in self.W]
        self.R = [colmajor(torch.zeros((w.shape[1], w.shape[1]), dtype=torch.float64, device=dev)) for w in self.W]
        self.info = torch.zeros((len(self.W), 4), dtype=torch.int32, device=dev)
        self.handle = rhqr_batch_create([sk.handle for sk in self.sketches], self.W, wt,
                                        [w.shape[0] for w in self.W], [w.shape[1] for w in self.W],
                                        [ld_of(w) for w in self.W], self.opts, self.Q, [ld_of(q) for q in self.Q],
                                        self.S, [ld_of(x) for x in self.S], self.T, self.R)
        self.ws_bytes = rhqr_batch_workspace_size(self.handle)
        self.ws = torch.empty(max(self.ws_bytes, 1), dtype=torch.uint8, device=dev)

    def close(self):
        if self.handle:
            rhqr_batch_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, stream=None):
        rhqr_factor_batched(self.handle, self.ws, self.ws_bytes, self.info, stream)

    def signature(self) -> str:
        """Autotuner cache key: device, dtype, passes and the problem shapes."""
        shapes = sorted((int(w.shape[0]), int(w.shape[1]), int(sk.k)) for sk, w in zip(self.sketches, self.W))
        import hashlib

        h = hashlib.sha1(repr(shapes).encode()).hexdigest()[:16]
        return f"{torch.cuda.get_device_name(self.W[0].device)}|{self.W[0].dtype}|p{self.opts.passes}|{h}"

    def tune(self, reps: int = 3, cache: str | None = None, stream=None) -> tuple:
        """Pick the launch shapes: from the JSON cache when it holds this
        signature, else by timing the candidates (and record them there)."""
        key = self.signature()
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
            if key in table:
                rhqr_batch_set_tuning(self.handle, table[key])
                return tuple(table[key])
        choice = rhqr_batch_tune(self.handle, self.ws, self.ws_bytes, self.info, reps, stream)
        if cache:
            table[key] = list(choice)
            with open(cache, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
        return choice

    def tuning(self) -> tuple:
        return rhqr_batch_get_tuning(self.handle)

    def capture(self):
        """A CUDA graph that replays the whole batch (one graph launch)."""
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(device=self.W[0].device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run(s)  # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(s)
        with torch.cuda.graph(g, stream=s):
            self.run(s)
        return g

    def infos(self) -> list[dict]:
        rows = self.info.cpu().tolist()
        return [dict(zip(("status", "column", "passes_done", "reserved"), r)) for r in rows]
