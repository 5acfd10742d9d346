"""Python binding of the GB300 randomized Householder QR library (C ABI in
``include/rhqr.h``).

This module only marshals arguments: every computation runs in the CUDA
kernels of ``_build/librhqr.so``.  Functions keep the C names.  Pointer
arguments accept either an integer device address or a torch tensor (its
``data_ptr()``); matrices are column-major, i.e. a torch tensor ``X`` of shape
(rows, cols) with ``X.stride(0) == 1`` and leading dimension ``X.stride(1)``
(see :func:`colmajor`).  There is no fallback: if the library is missing or
the GPU call fails, an exception is raised.
"""

from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

F64, F32, BF16, F16 = 0, 1, 2, 3
GAUSSIAN, SRHT = 0, 1
ALG_LEFT, ALG_REC, ALG_BLOCK = 0, 1, 2

STATUS = {
    0: "RHQR_OK",
    1: "RHQR_EINVAL",
    2: "RHQR_ENOMEM",
    3: "RHQR_ECUDA",
    4: "RHQR_EBREAKDOWN",
    5: "RHQR_ENONFINITE",
    6: "RHQR_ETIMEOUT",
    7: "RHQR_ENOTSUP",
}

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rhqr.h")


class RHQRError(RuntimeError):
    def __init__(self, func: str, code: int):
        self.code = code
        msg = f"{func} failed: {STATUS.get(code, code)}"
        if STATUS.get(code) == "RHQR_ECUDA":
            msg += " ({1}, code {0})".format(*rhqr_last_cuda_error())
        super().__init__(msg)


class rhqr_opts(ctypes.Structure):
    _fields_ = [
        ("alg", ctypes.c_int32),
        ("passes", ctypes.c_int32),
        ("limbs_first", ctypes.c_int32),
        ("limbs_refine", ctypes.c_int32),
        ("want_U", ctypes.c_int32),
        ("want_Q", ctypes.c_int32),
        ("scaling", ctypes.c_int32),
        ("solve", ctypes.c_int32),
        ("wait_budget", ctypes.c_int64),
        ("block_size", ctypes.c_int32),
        ("column_scaling", ctypes.c_int32),
    ]


class rhqr_info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("column", ctypes.c_int32),
        ("passes_done", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


_lib = None
_p = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_sz = ctypes.c_size_t

_SIGNATURES = {
    "rhqr_status_string": (ctypes.c_char_p, [_i32]),
    "rhqr_version": (_i32, []),
    "rhqr_built_arch": (_i32, []),
    "rhqr_default_opts": (None, [ctypes.POINTER(rhqr_opts)]),
    "rhqr_sketch_create": (_i32, [_i64, _i32, _i32, _u64, _i32, _p, ctypes.POINTER(_p)]),
    "rhqr_sketch_destroy": (_i32, [_p]),
    "rhqr_sketch_shape": (_i32, [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                 ctypes.POINTER(_i64), ctypes.POINTER(_i32)]),
    "rhqr_sketch_export": (_i32, [_p, _p, _p, _p, _i64, _p]),
    "rhqr_sketch_apply_workspace": (_i32, [_p, _i32, _i32, _i64, _i32, ctypes.POINTER(_sz)]),
    "rhqr_workspace_size": (_i32, [_p, _i64, _i32, _i32, ctypes.POINTER(rhqr_opts), ctypes.POINTER(_sz)]),
    "rhqr_sketch_apply": (_i32, [_p, _i32, _p, _i32, _i64, _i32, _i64, _p, _i64, _p, _sz, _p]),
    "rhqr_sketch_apply_rows_workspace": (_i32, [_p, _i32, _i32, _i64, _i64, _i32, ctypes.POINTER(_sz)]),
    "rhqr_sketch_apply_rows": (_i32, [_p, _i32, _p, _i32, _i64, _i64, _i32, _i64, _p, _i64, _p, _sz, _p]),
    "rhqr_factor": (_i32, [_p, _p, _i32, _i64, _i32, _i64, ctypes.POINTER(rhqr_opts), _p, _i64, _p, _i64, _p, _p,
                           _p, _i64, _p, _sz, _p, _p]),
    "rhqr_reconstruct": (_i32, [_p, _p, _i64, _p, _p, _p, _i64, _p, _i32, _i64, _i32, _i64, _p, _i64, _p, _i64, _p,
                                _sz, _p]),
    "rhqr_arnoldi_create": (_i32, [_p, _i64, _i32, _i32, _i32, ctypes.POINTER(_p)]),
    "rhqr_arnoldi_create_batch": (_i32, [_p, _i64, _i32, _i32, _i32, _i32, ctypes.POINTER(_p)]),
    "rhqr_stencil_apply": (_i32, [_i32, ctypes.c_double, _p, _i32, _i32, _p, _p]),
    "rhqr_stencil_residual_workspace": (_i32, [_i32, _i32, ctypes.POINTER(_sz)]),
    "rhqr_stencil_residual": (_i32, [_i32, ctypes.c_double, _p, _p, _i32, _i32, _p, _i32, _p, _p, _sz, _p]),
    "rhqr_arnoldi_solution_x": (_i32, [_p, _p, _i64, _i32, _p, _p, _p, _i32, _p, _p, _p]),
    "rhqr_arnoldi_destroy": (_i32, [_p]),
    "rhqr_arnoldi_begin": (_i32, [_p, _p, _p, _p, _p, _p]),
    "rhqr_arnoldi_step": (_i32, [_p, _p, _p, _p, _p, _p]),
    "rhqr_arnoldi_export": (_i32, [_p, _p, _i64, _p, _i64, _p, ctypes.POINTER(_i32), _p]),
    "rhqr_sketch_apply_noalloc": (_i32, [_p, _i32, _p, _i32, _i64, _i32, _i64, _p, _i64, _p]),
    "rhqr_arnoldi_solution": (_i32, [_p, _p, _i64, _i32, _p, _p, _p, _p, _p, _p]),
    "rhqr_blas2_rgs_workspace": (_i32, [_p, _i32, _i64, _i32, ctypes.POINTER(_sz)]),
    "rhqr_trim_workspace": (_i32, [_p, _i32, _i64, _i32, ctypes.POINTER(_sz)]),
    "rhqr_trim_factor": (_i32, [_p, _p, _i32, _i64, _i32, _i64, _i32, _p, _i64, _p, _i64, _p, _p, _p, _p, _i64, _p, _sz,
                                _p, _p]),
    "rhqr_blas2_rgs": (_i32, [_p, _p, _i32, _i64, _i32, _i64, _p, _i64, _p, _p, _p, _p, _sz, _p, _p]),
    "rhqr_batch_create": (_i32, [_i32, _p, _p, _i32, _p, _p, _p, ctypes.POINTER(rhqr_opts), _p, _p, _p, _p, _p, _p,
                                 ctypes.POINTER(_p)]),
    "rhqr_batch_workspace_size": (_i32, [_p, ctypes.POINTER(_sz)]),
    "rhqr_batch_destroy": (_i32, [_p]),
    "rhqr_factor_batched": (_i32, [_p, _p, _sz, _p, _p]),
    "rhqr_batch_tune": (_i32, [_p, _p, _sz, _p, _i32, _p, _p]),
    "rhqr_batch_get_tuning": (_i32, [_p, _p]),
    "rhqr_batch_set_tuning": (_i32, [_p, _p]),
    "rhqr_pipeline_create": (_i32, [_p, _i32, _i64, _i32, ctypes.POINTER(rhqr_opts), _i32, ctypes.POINTER(_p)]),
    "rhqr_pipeline_submit": (_i32, [_p, _p, _i64, _p, _i64, _p, _p, _i64, _p, _p]),
    "rhqr_pipeline_wait": (_i32, [_p]),
    "rhqr_pipeline_destroy": (_i32, [_p]),
    "rhqr_launch_count": (_i64, []),
    "rhqr_last_cuda_error": (_i32, []),
    "rhqr_cuda_error_name": (ctypes.c_char_p, [_i32]),
    "rhqr_profile_enable": (None, [_i32]),
    "rhqr_profile_read": (_i32, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64), _i32]),
}

PHASES = ["sketch", "hqr", "tfactor", "solve", "small", "left_step"]


def header_functions() -> list[str]:
    """Names of the functions declared in include/rhqr.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rhqr_[a-z0-9_]+)\s*\(", text)))


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first if needed) and bind the ABI."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError("CUDA library not built: call paper_2405_10923_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(name, code):
    if code != 0:
        raise RHQRError(name, code)


def colmajor(t, ld: int | None = None):
    """A column-major (Fortran-order) copy of a 2-D torch tensor, ld >= rows."""
    import torch

    rows, cols = t.shape
    ld = rows if ld is None else ld
    buf = torch.zeros((cols, ld), dtype=t.dtype, device=t.device)
    out = buf.t()[:rows]
    out.copy_(t)
    return out


def ld_of(t) -> int:
    if t.dim() != 2 or t.stride(0) != 1:
        raise ValueError("expected a column-major 2-D tensor (stride(0) == 1)")
    return max(t.stride(1), t.shape[0])


def dtype_code(t) -> int:
    import torch

    return {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}[t.dtype]


# ---------------------------------------------------------------------------
# the C entry points, same names
# ---------------------------------------------------------------------------


def rhqr_status_string(code: int) -> str:
    return load().rhqr_status_string(code).decode()


def rhqr_version() -> int:
    return load().rhqr_version()


def rhqr_built_arch() -> int:
    return load().rhqr_built_arch()


def rhqr_default_opts() -> rhqr_opts:
    o = rhqr_opts()
    load().rhqr_default_opts(ctypes.byref(o))
    return o


def rhqr_sketch_create(n: int, k: int, kind: int, seed: int, omega_dtype: int = F64, stream=None) -> int:
    out = _p()
    _check("rhqr_sketch_create",
           load().rhqr_sketch_create(n, k, kind, seed & ((1 << 64) - 1), omega_dtype, _stream(stream), ctypes.byref(out)))
    return out.value


def rhqr_sketch_destroy(s: int) -> None:
    _check("rhqr_sketch_destroy", load().rhqr_sketch_destroy(s))


def rhqr_sketch_shape(s: int):
    n, k, kind, N, dt = _i64(), _i32(), _i32(), _i64(), _i32()
    _check("rhqr_sketch_shape", load().rhqr_sketch_shape(s, ctypes.byref(n), ctypes.byref(k), ctypes.byref(kind),
                                                         ctypes.byref(N), ctypes.byref(dt)))
    return n.value, k.value, kind.value, N.value, dt.value


def rhqr_sketch_export(s: int, signs=None, rows=None, G=None, ldg: int = 0, stream=None) -> None:
    _check("rhqr_sketch_export", load().rhqr_sketch_export(s, _ptr(signs), _ptr(rows), _ptr(G), ldg, _stream(stream)))


def rhqr_sketch_apply_workspace(s: int, m: int, xt: int, n: int, c: int) -> int:
    b = _sz()
    _check("rhqr_sketch_apply_workspace", load().rhqr_sketch_apply_workspace(s, m, xt, n, c, ctypes.byref(b)))
    return b.value


def rhqr_workspace_size(s: int, n: int, m: int, wt: int, opts: rhqr_opts | None = None) -> int:
    b = _sz()
    _check("rhqr_workspace_size", load().rhqr_workspace_size(s, n, m, wt, ctypes.byref(opts) if opts else None,
                                                             ctypes.byref(b)))
    return b.value


def rhqr_sketch_apply(s, m, X, xt, n, c, ldx, Z, ldz, ws, ws_bytes, stream=None) -> None:
    _check("rhqr_sketch_apply", load().rhqr_sketch_apply(s, m, _ptr(X), xt, n, c, ldx, _ptr(Z), ldz, _ptr(ws),
                                                         ws_bytes, _stream(stream)))


def rhqr_arnoldi_create(s: int, n: int, mmax: int, basis_dtype: int = F64, scaling: int = 0) -> int:
    out = _p()
    _check("rhqr_arnoldi_create", load().rhqr_arnoldi_create(s, n, mmax, basis_dtype, scaling, ctypes.byref(out)))
    return out.value


def rhqr_arnoldi_create_batch(s: int, n: int, mmax: int, nrhs: int, basis_dtype: int = F64, scaling: int = 0) -> int:
    out = _p()
    _check("rhqr_arnoldi_create_batch",
           load().rhqr_arnoldi_create_batch(s, n, mmax, nrhs, basis_dtype, scaling, ctypes.byref(out)))
    return out.value


def rhqr_stencil_apply(g, pe, X, dt, nrhs, Y, stream=None) -> None:
    _check("rhqr_stencil_apply", load().rhqr_stencil_apply(g, pe, _ptr(X), dt, nrhs, _ptr(Y), _stream(stream)))


def rhqr_stencil_residual_workspace(g, nrhs) -> int:
    out = _sz()
    _check("rhqr_stencil_residual_workspace", load().rhqr_stencil_residual_workspace(g, nrhs, ctypes.byref(out)))
    return out.value


def rhqr_stencil_residual(g, pe, B, X, dt, nrhs, R, rdt, norms, work, work_bytes, stream=None) -> None:
    _check("rhqr_stencil_residual", load().rhqr_stencil_residual(g, pe, _ptr(B), _ptr(X), dt, nrhs, _ptr(R), rdt,
                                                                 _ptr(norms), _ptr(work), work_bytes,
                                                                 _stream(stream)))


def rhqr_arnoldi_solution_x(a, H, ldh, m, h0, x0, x, xdt, y, res, stream=None) -> None:
    _check("rhqr_arnoldi_solution_x", load().rhqr_arnoldi_solution_x(a, _ptr(H), ldh, m, _ptr(h0), _ptr(x0), _ptr(x),
                                                                     xdt, _ptr(y), _ptr(res), _stream(stream)))


def rhqr_arnoldi_destroy(a: int) -> None:
    _check("rhqr_arnoldi_destroy", load().rhqr_arnoldi_destroy(a))


def rhqr_arnoldi_begin(a, r0, h0, q1, info, stream=None) -> None:
    _check("rhqr_arnoldi_begin", load().rhqr_arnoldi_begin(a, _ptr(r0), _ptr(h0), _ptr(q1), _ptr(info),
                                                           _stream(stream)))


def rhqr_arnoldi_step(a, w, h, q_next, info, stream=None) -> None:
    _check("rhqr_arnoldi_step", load().rhqr_arnoldi_step(a, _ptr(w), _ptr(h), _ptr(q_next), _ptr(info),
                                                         _stream(stream)))


def rhqr_arnoldi_export(a, U=None, ldu=0, S=None, lds=0, T=None, stream=None) -> int:
    cnt = _i32()
    _check("rhqr_arnoldi_export", load().rhqr_arnoldi_export(a, _ptr(U), ldu, _ptr(S), lds, _ptr(T),
                                                             ctypes.byref(cnt), _stream(stream)))
    return cnt.value


def rhqr_arnoldi_solution(a, H, ldh, m, h0, x0, x, y, res, stream=None) -> None:
    _check("rhqr_arnoldi_solution", load().rhqr_arnoldi_solution(a, _ptr(H), ldh, m, _ptr(h0), _ptr(x0), _ptr(x),
                                                                 _ptr(y), _ptr(res), _stream(stream)))


def rhqr_blas2_rgs_workspace(s, wt, n, m) -> int:
    out = _sz()
    _check("rhqr_blas2_rgs_workspace", load().rhqr_blas2_rgs_workspace(s, wt, n, m, ctypes.byref(out)))
    return out.value


def rhqr_blas2_rgs(s, W, wt, n, m, ldw, Q, ldq, R, T, S, ws, ws_bytes, info, stream=None) -> None:
    _check("rhqr_blas2_rgs", load().rhqr_blas2_rgs(s, _ptr(W), wt, n, m, ldw, _ptr(Q), ldq, _ptr(R), _ptr(T), _ptr(S),
                                                   _ptr(ws), ws_bytes, _ptr(info), _stream(stream)))


def rhqr_sketch_apply_rows_workspace(s, m, xt, row0, rows, c) -> int:
    out = _sz()
    _check("rhqr_sketch_apply_rows_workspace",
           load().rhqr_sketch_apply_rows_workspace(s, m, xt, row0, rows, c, ctypes.byref(out)))
    return out.value


def rhqr_sketch_apply_rows(s, m, X, xt, row0, rows, c, ldx, Z, ldz, ws, ws_bytes, stream=None) -> None:
    _check("rhqr_sketch_apply_rows", load().rhqr_sketch_apply_rows(s, m, _ptr(X), xt, row0, rows, c, ldx, _ptr(Z), ldz,
                                                                   _ptr(ws), ws_bytes, _stream(stream)))


def rhqr_trim_workspace(s, wt, n, m) -> int:
    out = _sz()
    _check("rhqr_trim_workspace", load().rhqr_trim_workspace(s, wt, n, m, ctypes.byref(out)))
    return out.value


def rhqr_trim_factor(s, W, wt, n, m, ldw, scaling, U, ldu, S, lds, T, Tt, R, Q, ldq, ws, ws_bytes, info,
                     stream=None) -> None:
    _check("rhqr_trim_factor", load().rhqr_trim_factor(s, _ptr(W), wt, n, m, ldw, scaling, _ptr(U), ldu, _ptr(S), lds,
                                                       _ptr(T), _ptr(Tt), _ptr(R), _ptr(Q), ldq, _ptr(ws), ws_bytes,
                                                       _ptr(info), _stream(stream)))


def rhqr_sketch_apply_noalloc(s, m, X, xt, n, c, ldx, Z, ldz, stream=None) -> None:
    _check("rhqr_sketch_apply_noalloc", load().rhqr_sketch_apply_noalloc(s, m, _ptr(X), xt, n, c, ldx, _ptr(Z), ldz,
                                                                         _stream(stream)))


def _arr(ctype, values):
    return (ctype * len(values))(*values)


def rhqr_batch_create(sketches, W, wt, n, m, ldw, opts, Q, ldq, S, lds, T, R) -> int:
    """Plan over len(sketches) problems; every list holds one entry per problem
    (handles, ints, or tensors whose data pointers are taken)."""
    cnt = len(sketches)
    out = _p()
    _check("rhqr_batch_create", load().rhqr_batch_create(
        cnt, _arr(_p, sketches), _arr(_p, [_ptr(x) for x in W]), wt, _arr(_i64, n), _arr(_i32, m), _arr(_i64, ldw),
        ctypes.byref(opts) if opts else None, _arr(_p, [_ptr(x) for x in Q]), _arr(_i64, ldq),
        _arr(_p, [_ptr(x) for x in S]), _arr(_i64, lds), _arr(_p, [_ptr(x) for x in T]),
        _arr(_p, [_ptr(x) for x in R]), ctypes.byref(out)))
    return out.value


def rhqr_batch_workspace_size(b: int) -> int:
    out = _sz()
    _check("rhqr_batch_workspace_size", load().rhqr_batch_workspace_size(b, ctypes.byref(out)))
    return out.value


def rhqr_batch_destroy(b: int) -> None:
    _check("rhqr_batch_destroy", load().rhqr_batch_destroy(b))


def rhqr_factor_batched(b, ws, ws_bytes, info, stream=None) -> None:
    _check("rhqr_factor_batched", load().rhqr_factor_batched(b, _ptr(ws), ws_bytes, _ptr(info), _stream(stream)))


def rhqr_batch_tune(b, ws, ws_bytes, info, reps=3, stream=None) -> tuple:
    choice = (_i32 * 3)()
    _check("rhqr_batch_tune", load().rhqr_batch_tune(b, _ptr(ws), ws_bytes, _ptr(info), reps, choice,
                                                     _stream(stream)))
    return tuple(choice)


def rhqr_batch_get_tuning(b) -> tuple:
    choice = (_i32 * 3)()
    _check("rhqr_batch_get_tuning", load().rhqr_batch_get_tuning(b, choice))
    return tuple(choice)


def rhqr_batch_set_tuning(b, choice) -> None:
    _check("rhqr_batch_set_tuning", load().rhqr_batch_set_tuning(b, _arr(_i32, list(choice))))


def rhqr_factor(s, W, wt, n, m, ldw, opts, U, ldu, S, lds, T, R, Q, ldq, ws, ws_bytes, info, stream=None) -> None:
    _check("rhqr_factor", load().rhqr_factor(s, _ptr(W), wt, n, m, ldw, ctypes.byref(opts) if opts else None, _ptr(U),
                                             ldu, _ptr(S), lds, _ptr(T), _ptr(R), _ptr(Q), ldq, _ptr(ws), ws_bytes,
                                             _ptr(info), _stream(stream)))


def rhqr_reconstruct(s, S, lds, T, R, Z, ldz, W, wt, n, m, ldw, U, ldu, Q, ldq, ws, ws_bytes, stream=None) -> None:
    _check("rhqr_reconstruct", load().rhqr_reconstruct(s, _ptr(S), lds, _ptr(T), _ptr(R), _ptr(Z), ldz, _ptr(W), wt, n,
                                                       m, ldw, _ptr(U), ldu, _ptr(Q), ldq, _ptr(ws), ws_bytes,
                                                       _stream(stream)))


def rhqr_pipeline_create(s, wt, n, m, opts, depth=2) -> int:
    out = _p()
    _check("rhqr_pipeline_create", load().rhqr_pipeline_create(s, wt, n, m, ctypes.byref(opts) if opts else None, depth,
                                                               ctypes.byref(out)))
    return out.value


def rhqr_pipeline_submit(p, W, ldw, Q, ldq, R, S=None, lds=0, T=None, info=None) -> None:
    """W, Q, R, S, T, info: host buffers (CPU tensors or addresses)."""
    _check("rhqr_pipeline_submit", load().rhqr_pipeline_submit(p, _ptr(W), ldw, _ptr(Q), ldq, _ptr(R), _ptr(S), lds,
                                                               _ptr(T), _ptr(info)))


def rhqr_pipeline_wait(p) -> None:
    _check("rhqr_pipeline_wait", load().rhqr_pipeline_wait(p))


def rhqr_pipeline_destroy(p) -> None:
    _check("rhqr_pipeline_destroy", load().rhqr_pipeline_destroy(p))


def rhqr_launch_count() -> int:
    return load().rhqr_launch_count()


def rhqr_last_cuda_error() -> tuple[int, str]:
    """CUDA error code and name of the last call that returned RHQR_ECUDA (0 if none)."""
    code = load().rhqr_last_cuda_error()
    return code, load().rhqr_cuda_error_name(code).decode()


def rhqr_profile_enable(on: bool) -> None:
    load().rhqr_profile_enable(1 if on else 0)


def rhqr_profile_read() -> dict:
    """{phase: (milliseconds, calls)} for the phases recorded since enabling."""
    n = len(PHASES)
    ms = (ctypes.c_double * n)()
    calls = (_i64 * n)()
    load().rhqr_profile_read(ms, calls, n)
    return {PHASES[i]: (ms[i], int(calls[i])) for i in range(n)}


def read_info(info_tensor) -> dict:
    """Decode a 4-int32 device tensor holding an rhqr_info (synchronises).  For
    several records (an (r, 4) tensor) the first non-OK one is returned (the
    first one when all are OK)."""
    rows = info_tensor.reshape(-1, 4).cpu().tolist()
    v = next((r for r in rows if r[0] != 0), rows[0])
    return {"status": int(v[0]), "column": int(v[1]), "passes_done": int(v[2])}
