"""BLAS2-RGS (Algorithm 9) on the GPU against the oracle's blas2_rgs with the
same Omega_full (Gaussian float64 operator and SRHT): Q, R, T and S = Omega Q
agree to rounding; W = Q R and Omega Q is orthonormal."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import rhqr_inputs as ri  # noqa: E402
from oracle import rhqr, sketch  # noqa: E402


@pytest.mark.parametrize("kind,n,m,k", [("gaussian", 3000, 12, 64), ("srht", 2500, 9, 48), ("srht", 4096, 24, 96)])
def test_blas2_rgs_matches_oracle(gpu_lib, kind, n, m, k):
    from paper_2405_10923_gb300 import torch_api as ta

    W = ri.spectrum(n, m, 1e6, 61)
    if kind == "gaussian":
        sk, osk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, 62, gpu_lib.F64), sketch.GaussianSketch(n, k, 62, "f64")
    else:
        sk, osk = ta.Sketch(n, k, gpu_lib.SRHT, 62), sketch.SRHTSketch(n, k, 62)
    Om = np.asarray(osk.full_matrix())[:, :n]
    Qo, Ro, So, To = rhqr.blas2_rgs(W, Om)
    Q, R, T, S, info = ta.blas2_rgs(sk, gpu_lib.colmajor(torch.tensor(W, device="cuda")))
    torch.cuda.synchronize()
    assert gpu_lib.read_info(info)["status"] == 0
    Q, R, T, S = (x.cpu().numpy() for x in (Q, R, T, S))
    assert np.max(np.abs(R - Ro)) <= 1e-11 * np.abs(Ro).max()
    assert np.max(np.abs(Q - Qo)) <= 1e-10 * np.abs(Qo).max()
    assert np.max(np.abs(T - To)) <= 1e-9
    assert np.max(np.abs(S - So)) <= 1e-10
    assert np.max(np.abs(W - Q @ R)) <= 1e-12 * np.abs(W).max()
    assert np.max(np.abs(S.T @ S - np.eye(m))) <= 1e-9
    sk.close()


def test_blas2_rgs_float32(gpu_lib):
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 3000, 10, 64
    W = ri.gaussian(n, m, 63)
    sk, osk = ta.Sketch(n, k, gpu_lib.SRHT, 64), sketch.SRHTSketch(n, k, 64)
    Qo, Ro, _, _ = rhqr.blas2_rgs(W, np.asarray(osk.full_matrix())[:, :n])
    Q, R, T, S, info = ta.blas2_rgs(sk, gpu_lib.colmajor(torch.tensor(W, dtype=torch.float32, device="cuda")))
    torch.cuda.synchronize()
    assert gpu_lib.read_info(info)["status"] == 0
    assert np.max(np.abs(R.cpu().numpy() - Ro)) <= 1e-5 * np.abs(Ro).max()
    assert np.max(np.abs(Q.double().cpu().numpy() - Qo)) <= 1e-5 * np.abs(Qo).max()
    sk.close()


def test_blas2_rgs_rejects_more_columns_than_sketch_rows(gpu_lib):
    """Omega Q (k x m) cannot have orthonormal columns when m > k: the call is
    an argument error, reported before any device work."""
    from paper_2405_10923_gb300 import torch_api as ta

    n, k = 1000, 8
    sk = ta.Sketch(n, k, gpu_lib.SRHT, 63)
    assert gpu_lib.rhqr_blas2_rgs_workspace(sk.handle, gpu_lib.F64, n, k) > 0
    with pytest.raises(gpu_lib.RHQRError) as e:
        gpu_lib.rhqr_blas2_rgs_workspace(sk.handle, gpu_lib.F64, n, k + 1)
    assert e.value.code == 1  # RHQR_EINVAL
    sk.close()
