"""blockRHQR (Algorithm 5) on the GPU against the oracle's block_rhqr.

Float64: U, S = Psi U, R and each block's T^(j) (the diagonal blocks of the
returned T) agree with the oracle to 1e-11 relative, over ragged last blocks,
one-block and one-column-block cases, Gaussian and SRHT sketches.  In exact
arithmetic the reflectors are those of left-looking RHQR on the whole W, so
the returned compact-form T (from the Woodbury identity) and Q agree with the
oracle's rhqr_left to the same tolerance.  Float32 keeps the stated 1e-5 on
||I - (Psi Q)^t Psi Q||_2 and ||W - QR||_F / ||W||_F at cond 1e10 (the
condition-number independence of RHQR)."""

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


def _sketches(gpu_lib, kind, n, k, seed):
    from paper_2405_10923_gb300 import torch_api as ta

    if kind == "srht":
        return ta.Sketch(n, k, gpu_lib.SRHT, seed), sketch.SRHTSketch(n, k, seed)
    return ta.Sketch(n, k, gpu_lib.GAUSSIAN, seed), sketch.GaussianSketch(n, k, seed)


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
@pytest.mark.parametrize("n,m,k,bs", [(3000, 40, 96, 16), (2500, 24, 64, 8), (4096, 33, 128, 32), (1500, 12, 48, 64),
                                      (1200, 7, 24, 1)])
def test_block_rhqr_f64_matches_oracle(gpu_lib, kind, n, m, k, bs):
    from paper_2405_10923_gb300 import torch_api as ta

    W = ri.gaussian(n, m, 70)
    sk, osk = _sketches(gpu_lib, kind, n, k, 71)
    out = ta.factor(sk, _dev(W), alg=gpu_lib.ALG_BLOCK, block_size=bs)
    torch.cuda.synchronize()
    assert ta.info(out)["status"] == 0
    R_o, blocks = rhqr.block_rhqr(W, osk, bs)
    R, U, S, T = _np(out["R"]), _np(out["U"]), _np(out["S"]), _np(out["T"])
    tol = 1e-11
    assert np.max(np.abs(R - R_o)) <= tol * np.abs(R_o).max()
    for c0, Uj, Sj, Tj in blocks:
        c1 = c0 + Uj.shape[1]
        assert np.max(np.abs(U[:, c0:c1] - Uj)) <= tol * max(1, np.abs(Uj).max())
        assert np.max(np.abs(S[:, c0:c1] - Sj)) <= tol * max(1, np.abs(Sj).max())
        assert np.max(np.abs(T[c0:c1, c0:c1] - Tj)) <= tol * max(1, np.abs(Tj).max())
    # the same reflectors as Algorithm 4 on the whole W: full T and Q
    U_l, S_l, T_l, R_l = rhqr.rhqr_left(W, osk)
    assert np.max(np.abs(T - T_l)) <= tol * max(1, np.abs(T_l).max())
    assert np.max(np.abs(_np(out["Q"]) - rhqr.form_q(U_l, T_l))) <= tol
    sk.close()


@pytest.mark.parametrize("cond", [1e4, 1e10])
def test_block_rhqr_f32_invariants(gpu_lib, cond):
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 1 << 16, 64, 256
    W = ri.spectrum(n, m, cond, 72).astype(np.float32).astype(np.float64)
    sk, osk = _sketches(gpu_lib, "srht", n, k, 73)
    out = ta.factor(sk, _dev(W, torch.float32), alg=gpu_lib.ALG_BLOCK, block_size=16)
    torch.cuda.synchronize()
    assert ta.info(out)["status"] == 0
    Q, R = _np(out["Q"]), _np(out["R"])
    assert metrics.sketch_orthogonality(Q, osk) <= 1e-5
    assert metrics.residual(W, Q, R) <= 1e-5
    sk.close()


def test_block_rhqr_rejects_bad_block_size(gpu_lib):
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 1000, 8, 32
    sk = ta.Sketch(n, k, gpu_lib.SRHT, 74)
    for bs in (0, 65):
        with pytest.raises(gpu_lib.RHQRError) as e:
            ta.factor(sk, _dev(ri.gaussian(n, m, 75)), alg=gpu_lib.ALG_BLOCK, block_size=bs)
        assert e.value.code == 1
    sk.close()
