"""Left-looking trimRHQR (Section 7) on the GPU against the oracle's trim_rhqr_left.

The oracle takes Omega as an explicit k x n matrix with unit first m columns:
the SRHT's Omega_full has them (k entries +-1/sqrt(k) per column); for a
Gaussian sketch the library normalises the first m columns of Omega_full, and
the test hands the oracle that same matrix.  Float64: U, S = Omega U, T, Tt
and R agree to 1e-11 relative, including sketch sizes k smaller than m (the
case the section is written for), both reflector scalings, and Q agrees with
[I; 0] - U T ut((Omega U)^t Omega)[I; 0] built by the oracle; W = QR holds to
rounding.  Float32 keeps ||W - QR||_F / ||W||_F within the stated 1e-5."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import rhqr_inputs as ri  # noqa: E402
from oracle import metrics, rhqr, sketch  # noqa: E402


def _dev(W, dtype=torch.float64):
    import paper_2405_10923_gb300 as rh

    return rh.colmajor(torch.tensor(W, dtype=dtype, device="cuda"))


def _np(t):
    return t.detach().double().cpu().numpy()


def _omega(gpu_lib, kind, n, m, k, seed):
    from paper_2405_10923_gb300 import torch_api as ta

    if kind == "srht":
        sk = ta.Sketch(n, k, gpu_lib.SRHT, seed)
        om = np.asarray(sketch.SRHTSketch(n, k, seed).full_matrix())[:, :n]
    else:
        sk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, seed)
        om = np.array(sketch.GaussianSketch(n, k, seed).full_matrix())
        om[:, :m] /= np.linalg.norm(om[:, :m], axis=0)[None, :]
    return sk, om


def _close(a, b, tol):
    return np.max(np.abs(a - b)) <= tol * max(1.0, np.abs(b).max())


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
@pytest.mark.parametrize("n,m,k", [(2000, 16, 48), (3000, 40, 24), (1500, 12, 8), (4099, 33, 64)])
@pytest.mark.parametrize("scaling", [0, 1])
def test_trim_rhqr_f64_matches_oracle(gpu_lib, kind, n, m, k, scaling):
    from paper_2405_10923_gb300 import torch_api as ta

    W = ri.gaussian(n, m, 90)
    sk, om = _omega(gpu_lib, kind, n, m, k, 91)
    out = ta.trim_factor(sk, _dev(W), scaling=scaling)
    torch.cuda.synchronize()
    assert ta.read_info(out["info"])["status"] == 0
    U, S, T, Tt, R = rhqr.trim_rhqr_left(W, om, scaling="unit" if scaling == 0 else "norm")
    tol = 1e-11
    assert np.max(np.abs(_np(out["R"]) - R)) <= tol * np.abs(R).max()
    assert _close(_np(out["U"]), U, tol)
    assert _close(_np(out["S"]), S, tol)
    assert _close(_np(out["T"]), T, tol)
    assert _close(_np(out["Tt"]), Tt, tol)
    top = np.zeros((n, m))
    top[np.arange(m), np.arange(m)] = 1.0
    Qo = top - U @ (T @ rhqr.trim_ut(S, om, top))
    Q = _np(out["Q"])
    assert np.max(np.abs(Q - Qo)) <= tol * max(1.0, np.abs(Qo).max())
    assert metrics.residual(W, Q, _np(out["R"])) <= 1e-13
    sk.close()


@pytest.mark.parametrize("cond", [1e4, 1e8])
def test_trim_rhqr_f32_factorisation(gpu_lib, cond):
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 1 << 16, 64, 48  # fewer sketch rows than columns
    W = ri.spectrum(n, m, cond, 92).astype(np.float32).astype(np.float64)
    sk = ta.Sketch(n, k, gpu_lib.SRHT, 93)
    out = ta.trim_factor(sk, _dev(W, torch.float32))
    torch.cuda.synchronize()
    assert ta.read_info(out["info"])["status"] == 0
    Q, R = _np(out["Q"]), _np(out["R"])
    assert metrics.residual(W, Q, R) <= 1e-5
    sk.close()
