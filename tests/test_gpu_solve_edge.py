"""Edge cases of recRHQR's row solve Q = W R^{-1} (Section 3.3) in float32.

The default solve multiplies by the explicit inverse R^{-1} = D (I + F) on
the tensor cores; the alternative (opts.solve = 1) runs a row-wise
substitution.  A product with an explicit inverse is not backward stable in
general, and the inputs where it is most likely to lose against substitution
are those whose R is strongly graded: W with column norms spread over ten
orders of magnitude, and W = Q0 R0 with R0 = D0 (I + E) for a graded diagonal
D0.  For both solves, one pass and three passes, the factorisation error
||W - QR||_F / ||W||_F must stay at the float32 tolerance (1e-5), and after
three passes the sketch orthogonality ||I - (Psi Q)^t Psi Q||_2 as well, both
measured with the oracle's FP64 sketch.  The one-pass R is also compared with
the oracle's recRHQR R: the GPU sketches float32 data with the SRHT in float32
arithmetic, whose error is at most gamma_{log2 N + 5} of float32 relative to
each column (the SRHT error lemma of Section 4), about 1.2e-6 for N = 2^15;
the Householder QR of the sketch passes that on to R column by column.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import rhqr_inputs as ri  # noqa: E402
from oracle import metrics, rhqr, sketch  # noqa: E402

N, M, K = 1 << 15, 256, 512


def _graded_columns(seed):
    G = ri.gaussian(N, M, seed)
    return G * np.logspace(0.0, -10.0, M)[None, :]


def _graded_r(seed):
    rng = np.random.default_rng(seed)
    Q0 = ri.orthonormal(N, M, rng)
    E = np.triu(rng.standard_normal((M, M)), 1) / np.sqrt(M)
    R0 = np.logspace(0.0, -10.0, M)[:, None] * (np.eye(M) + E)
    return Q0 @ R0


INPUTS = {"graded_columns": _graded_columns, "graded_r": _graded_r}


@pytest.mark.parametrize("solve", [0, 1])
@pytest.mark.parametrize("passes", [1, 3])
@pytest.mark.parametrize("kind", sorted(INPUTS))
def test_graded_inputs(gpu_lib, kind, passes, solve):
    import paper_2405_10923_gb300 as rh
    from paper_2405_10923_gb300 import torch_api as ta

    W = INPUTS[kind](40).astype(np.float32).astype(np.float64)
    sk, osk = ta.Sketch(N, K, gpu_lib.SRHT, 41), sketch.SRHTSketch(N, K, 41)
    Wd = rh.colmajor(torch.tensor(W, dtype=torch.float32, device="cuda"))
    out = ta.factor(sk, Wd, alg=gpu_lib.ALG_REC, passes=passes, solve=solve)
    torch.cuda.synchronize()
    assert ta.info(out)["status"] == 0
    Q, R = out["Q"].double().cpu().numpy(), out["R"].cpu().numpy()
    resid = metrics.residual(W, Q, R)
    assert resid <= 1e-5, resid
    if passes == 3:
        assert metrics.sketch_orthogonality(Q, osk) <= 1e-5
    else:
        _U, _S, _T, Ro, _M = rhqr.rec_rhqr(W, osk)
        u32 = 2.0**-24
        gamma = (15 + 5) * u32 / (1 - (15 + 5) * u32)
        assert metrics.r_relative_difference(R, Ro) <= gamma
    sk.close()
