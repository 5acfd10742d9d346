"""Tensor-core (tcgen05) Gaussian sketch and the mixed-precision recRHQR path,
against the FP64 oracle using the same 16-bit Gaussian operator.

Tolerances: the 3-limb split represents float32 data exactly, so the only
error is the float32 accumulation inside a K-chunk of 8192 rows:
|Z - Z_oracle| <= 2e-5 max|Z_oracle|.  The factorisation tolerances are the
stated ones: <= 5e-3 before refinement (one bf16 limb, well-conditioned W) and
<= 1e-5 after refinement for ||I - (Psi Q)^t Psi Q||_2 and ||W - QR||/||W||."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import rhqr_inputs as ri  # noqa: E402
from oracle import metrics, rhqr, sketch  # noqa: E402


def _dev(W, dtype=torch.float32):
    import paper_2405_10923_gb300 as rh

    return rh.colmajor(torch.tensor(W, dtype=dtype, device="cuda"))


def _np(t):
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("dt", ["bf16", "f16"])
@pytest.mark.parametrize("n,m,c,k", [(50000, 16, 16, 1024), (40003, 13, 40, 300), (70000, 256, 256, 512),
                                     (9000, 0, 7, 256), (20000, 5, 256, 1024), (30001, 100, 100, 256),
                                     (12345, 70, 129, 640)])
def test_tc_sketch_matches_oracle(gpu_lib, dt, n, m, c, k):
    from paper_2405_10923_gb300 import torch_api as ta

    code = gpu_lib.BF16 if dt == "bf16" else gpu_lib.F16
    X = ri.gaussian(n, c, 70).astype(np.float32).astype(np.float64)
    sk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, 71, code)
    Z = _np(sk.apply(_dev(X), m))
    Zo = sketch.rh_sketch(X, m, sketch.GaussianSketch(n, k, 71, dt))
    assert np.array_equal(Z[:m], Zo[:m])
    assert np.max(np.abs(Z - Zo)) <= 2e-5 * np.abs(Zo).max()
    sk.close()


def _orth_exact(gpu_lib, sk, Q, m):
    """||I - (Psi Q)^t Psi Q||_2 with Psi Q accumulated in float64 on the GPU
    (the same stored operator, the SIMT float64 path)."""
    Z = sk.apply(Q.double().contiguous().t().contiguous().t(), m)
    G = (Z.t() @ Z).cpu().numpy()
    return float(np.max(np.abs(np.linalg.eigvalsh(np.eye(G.shape[0]) - G))))


@pytest.mark.parametrize("m,limbs", [(64, 1), (160, 1), (256, 2)])
def test_mixed_rec_one_pass_well_conditioned(gpu_lib, m, limbs):
    """m > 128: two column tiles of X, sketched on CTA pairs (cta_group::2).
    One bf16 limb of X at m = 256 gives orth ~5.6e-3 (above the one-pass 5e-3):
    the 256-column case takes the two limbs of the default options."""
    from paper_2405_10923_gb300 import torch_api as ta

    n, k = 1 << 17, 512
    W = ri.gaussian(n, m, 80).astype(np.float32).astype(np.float64)
    sk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, 81, gpu_lib.BF16)
    out = ta.factor(sk, _dev(W), alg=gpu_lib.ALG_REC, passes=1, limbs_first=limbs)
    torch.cuda.synchronize()
    assert ta.info(out)["status"] == 0
    osk = sketch.GaussianSketch(n, k, 81, "bf16")
    Q = _np(out["Q"])
    assert metrics.sketch_orthogonality(Q, osk) <= 5e-3
    assert metrics.residual(W, Q, _np(out["R"])) <= 1e-5
    sk.close()


@pytest.mark.parametrize("dt", ["bf16", "f16"])
@pytest.mark.parametrize("cond", [1e4, 1e10])
def test_mixed_rec_refined_meets_tolerance(gpu_lib, cond, dt):
    """bf16 and fp16 operators.  The fp16 limbs of X are taken after an exact
    power-of-two scaling of each column (fp16's narrow exponent range would
    otherwise push the lower limbs of entries ~1/sqrt(n) into subnormals)."""
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 1 << 17, 64, 256
    W = ri.spectrum(n, m, cond, 82).astype(np.float32).astype(np.float64)
    sk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, 83, gpu_lib.BF16 if dt == "bf16" else gpu_lib.F16)
    out = ta.factor(sk, _dev(W), alg=gpu_lib.ALG_REC, passes=3, limbs_first=2, limbs_refine=2)
    torch.cuda.synchronize()
    assert ta.info(out)["status"] == 0 and ta.info(out)["passes_done"] == 3
    osk = sketch.GaussianSketch(n, k, 83, dt)
    Q = _np(out["Q"])
    assert metrics.sketch_orthogonality(Q, osk) <= 1e-5
    assert metrics.residual(W, Q, _np(out["R"])) <= 1e-5
    sk.close()


# ---------------------------------------------------------------------------
# tensor-core row solve Q = W R^{-1} (float32 data, m <= 256)
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("solve", [0, 1])
@pytest.mark.parametrize("n,m", [(5000, 256), (4099, 200), (3000, 130), (2000, 64), (2500, 65), (1000, 17),
                                 (70001, 256), (300, 1), (127, 16), (20000, 161), (9000, 176), (6000, 255),
                                 (1025, 160)])
def test_tc_solve_matches_oracle(gpu_lib, n, m, solve):
    """Both float32 tensor-core solves (explicit-inverse product, row-wise
    substitution) over column counts that exercise one or two CTAs per row
    tile, partial 16-column groups and row tiles smaller than 128."""
    from paper_2405_10923_gb300 import torch_api as ta

    k = max(2 * m, 64)
    W = ri.gaussian(n, m, 90).astype(np.float32).astype(np.float64)
    sk, osk = ta.Sketch(n, k, gpu_lib.SRHT, 91), sketch.SRHTSketch(n, k, 91)
    out = ta.factor(sk, _dev(W), alg=gpu_lib.ALG_REC, passes=1, solve=solve)
    torch.cuda.synchronize()
    assert ta.info(out)["status"] == 0
    Q, R = _np(out["Q"]), _np(out["R"])
    # backward stable row solves: residual at float32 level
    assert metrics.residual(W, Q, R) <= 1e-6
    U, S, T, Ro, M = rhqr.rec_rhqr(W, osk)
    assert np.max(np.abs(Q - rhqr.form_q(U, T))) <= 1e-4
    assert metrics.sketch_orthogonality(Q, osk) <= 1e-5
    sk.close()


@pytest.mark.parametrize("solve", [0, 1])
def test_tc_solve_in_place_refinement_high_condition(gpu_lib, solve):
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 1 << 16, 256, 512
    W = ri.spectrum(n, m, 1e8, 92).astype(np.float32).astype(np.float64)
    sk, osk = ta.Sketch(n, k, gpu_lib.SRHT, 93), sketch.SRHTSketch(n, k, 93)
    out = ta.factor(sk, _dev(W), alg=gpu_lib.ALG_REC, passes=3, solve=solve)
    torch.cuda.synchronize()
    assert ta.info(out)["passes_done"] == 3
    Q, R = _np(out["Q"]), _np(out["R"])
    assert metrics.residual(W, Q, R) <= 1e-5
    assert metrics.sketch_orthogonality(Q, osk) <= 1e-5
    sk.close()


def test_tc_factor_repeatable_bitwise(gpu_lib):
    """Every kernel of the float32 path is deterministic (fixed-order reductions,
    no atomics on data): repeated factorisations of the same W give the same
    bits.  A stage of a TMA pipeline released before its shared-memory reads had
    completed once let a refill overwrite a tile's data; this repeats the
    factorisation enough times to catch such a race."""
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 1 << 21, 256, 1024
    W = ri.device_spectrum(n, m, 1e10, 94)
    sk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, 95, gpu_lib.BF16)
    out = ta.factor(sk, W, alg=gpu_lib.ALG_REC, passes=3)
    ws = out["ws"]
    torch.cuda.synchronize()
    Q0, R0 = out["Q"].clone(), out["R"].clone()
    for _ in range(12):
        ta.factor(sk, W, alg=gpu_lib.ALG_REC, passes=3, out=out, ws=ws)
        torch.cuda.synchronize()
        assert torch.equal(out["Q"], Q0) and torch.equal(out["R"], R0)
    sk.close()
