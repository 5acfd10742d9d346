"""The allocation-free sketch entry point (for callers that cannot allocate
device memory when they call: framework hooks that forbid it, real-time paths
that must not wait on the allocator, hosts that own all device memory) against
the workspace entry point, through the C ABI, on two calls in a row.  Both run
the same kernels with the same work split (it depends on the shapes only), so
the results must agree bit for bit; a stale or shared-scratch contamination
would show.  This file is collected last so that a run stopping at the first
failure has already run every other test."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import rhqr_inputs as ri  # noqa: E402


@pytest.mark.parametrize("kind,dt,n,m,c,k", [("gaussian", "bf16", 50000, 16, 64, 1024),
                                             ("gaussian", "f64", 20000, 8, 12, 256),
                                             ("srht", "f64", 100000, 5, 7, 512)])
def test_noalloc_matches_workspace_entry(gpu_lib, kind, dt, n, m, c, k):
    rh = gpu_lib
    from paper_2405_10923_gb300 import torch_api as ta

    code = {"bf16": rh.BF16, "f64": rh.F64}[dt]
    sk = ta.Sketch(n, k, rh.GAUSSIAN if kind == "gaussian" else rh.SRHT, 5, code)
    xdt = torch.float32 if dt == "bf16" else torch.float64
    X = rh.colmajor(torch.tensor(ri.gaussian(n, c, 6), dtype=xdt, device="cuda"))
    Zref = sk.apply(X, m).cpu().numpy()
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        Z = rh.colmajor(torch.full((k + m, c), np.nan, dtype=torch.float64, device="cuda"))
        rh.rhqr_sketch_apply_noalloc(sk.handle, m, X, rh.dtype_code(X), n, c, rh.ld_of(X), Z, rh.ld_of(Z))
        Zn = Z.cpu().numpy()
        # same kernels, work split and reduction order: identical bits
        assert np.array_equal(Zn, Zref)
    sk.close()


def test_noalloc_rejects_oversized_requests(gpu_lib):
    rh = gpu_lib
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, c, k = 1 << 16, 0, 256, 8192  # SRHT stage buffer c * (N/8192) * d2 * 8 bytes > scratch
    sk = ta.Sketch(n, k, rh.SRHT, 7)
    X = rh.colmajor(torch.zeros((n, c), dtype=torch.float64, device="cuda"))
    Z = rh.colmajor(torch.zeros((k + m, c), dtype=torch.float64, device="cuda"))
    need = rh.rhqr_sketch_apply_workspace(sk.handle, m, rh.F64, n, c)
    assert need > 24 * 1024 * 1024
    with pytest.raises(rh.RHQRError) as e:
        rh.rhqr_sketch_apply_noalloc(sk.handle, m, X, rh.F64, n, c, n, Z, k + m)
    assert e.value.code == 2  # RHQR_ENOMEM
    sk.close()
