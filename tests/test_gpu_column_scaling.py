"""rhqr_opts.column_scaling: each recRHQR pass equilibrates the columns of its
sketch Z before the Householder QR and multiplies them back into R.  The
Householder QR of Z D^{-1} has the reflectors of Z and the R factor R D^{-1}
(Section 3.3 with Psi W D^{-1}), so the factors must agree with the oracle's
recRHQR of W itself -- column by column of R, whose columns here span 24
orders of magnitude -- and the float32 mixed path must meet the stated 1e-5."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import rhqr_inputs as ri  # noqa: E402
from oracle import metrics, rhqr, sketch  # noqa: E402


def _colwise(R, Ro):
    return max(np.linalg.norm(R[:, j] - Ro[:, j]) / np.linalg.norm(Ro[:, j]) for j in range(R.shape[1]))


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
def test_column_scaling_f64_matches_oracle(gpu_lib, kind):
    import paper_2405_10923_gb300 as rh
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 4000, 24, 96
    W = ri.gaussian(n, m, 80) * np.logspace(-12, 12, m)[None, :]
    if kind == "srht":
        sk, osk = ta.Sketch(n, k, gpu_lib.SRHT, 81), sketch.SRHTSketch(n, k, 81)
    else:
        sk, osk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, 81), sketch.GaussianSketch(n, k, 81)
    Wd = rh.colmajor(torch.tensor(W, device="cuda"))
    out = ta.factor(sk, Wd, alg=gpu_lib.ALG_REC, column_scaling=1, want_U=True)
    torch.cuda.synchronize()
    assert ta.info(out)["status"] == 0
    U, S, T, Ro, M = rhqr.rec_rhqr(W, osk)
    R = out["R"].cpu().numpy()
    assert _colwise(R, Ro) <= 1e-11
    assert np.max(np.abs(out["S"].cpu().numpy() - S)) <= 1e-11
    assert np.max(np.abs(out["T"].cpu().numpy() - T)) <= 1e-11 * max(1, np.abs(T).max())
    assert metrics.sketch_orthogonality(out["Q"].cpu().numpy(), osk) <= 1e-12
    sk.close()


def test_column_scaling_mixed_path_meets_tolerance(gpu_lib):
    import paper_2405_10923_gb300 as rh
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 1 << 16, 64, 256
    W = (ri.spectrum(n, m, 1e6, 82) * np.logspace(-15, 15, m)[None, :]).astype(np.float32).astype(np.float64)
    sk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, 83, gpu_lib.BF16)
    out = ta.factor(sk, rh.colmajor(torch.tensor(W, dtype=torch.float32, device="cuda")), alg=gpu_lib.ALG_REC,
                    passes=3, column_scaling=1)
    torch.cuda.synchronize()
    assert ta.info(out)["status"] == 0
    osk = sketch.GaussianSketch(n, k, 83, "bf16")
    Q, R = out["Q"].double().cpu().numpy(), out["R"].cpu().numpy()
    assert metrics.sketch_orthogonality(Q, osk) <= 1e-5
    assert metrics.residual(W, Q, R) <= 1e-5
    sk.close()
