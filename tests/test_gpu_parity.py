"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (float64 data): entries of U, S, T, R, Q agree to 1e-11 relative
(well-conditioned inputs, so the factors are unique and stable);
||I - (Psi Q)^t Psi Q||_2 and ||W - QR||_F/||W||_F <= 1e-12.  Float32 data:
<= 1e-5 (the FP32 path's stated bound).  Integer work (signs, sampled rows)
and the Gaussian entries (same formula, correctly rounded operations only)
are compared bit for bit."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import rhqr_inputs as ri  # noqa: E402
from oracle import metrics, rhqr, rng, sketch  # noqa: E402


def _dev(W, dtype=None):
    import paper_2405_10923_gb300 as rh

    t = torch.tensor(W, dtype=dtype or torch.float64, device="cuda")
    return rh.colmajor(t)


def _np(t):
    return t.detach().double().cpu().numpy()


# ---------------------------------------------------------------------------
# random operators: bit exact
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("n,k,seed", [(64, 8, 1), (1000, 100, 2), (5000, 512, 3), (1 << 20, 512, 2002), (300000, 400, 5)])
def test_srht_signs_and_rows_bit_exact(gpu_lib, n, k, seed):
    from paper_2405_10923_gb300 import torch_api as ta

    sk = ta.Sketch(n, k, gpu_lib.SRHT, seed)
    ex = sk.export()
    N = sketch.next_pow2(n)
    assert sk.N == N
    assert np.array_equal(ex["signs"].cpu().numpy().astype(np.float64), rng.srht_signs(seed, N))
    assert np.array_equal(ex["rows"].cpu().numpy().astype(np.int64), rng.srht_sample(seed, N, k))
    sk.close()


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16", "f16"])
def test_gaussian_entries_bit_exact(gpu_lib, dt):
    from paper_2405_10923_gb300 import torch_api as ta

    code = {"f64": gpu_lib.F64, "f32": gpu_lib.F32, "bf16": gpu_lib.BF16, "f16": gpu_lib.F16}[dt]
    n, k, seed = 777, 40, 11
    sk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, seed, code)
    G = _np(sk.export()["G"])
    want = rng.gaussian_block(seed, n, np.arange(k), np.arange(n), dt)
    assert np.array_equal(G, want)
    sk.close()


def test_gaussian_entries_sampled_at_full_size(gpu_lib):
    # the operator of the 2^22 x 256 workload (k = 1024, bf16), checked at sampled entries
    from paper_2405_10923_gb300 import torch_api as ta

    n, k, seed = 1 << 22, 1024, 2003
    sk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, seed, gpu_lib.BF16)
    G = sk.export()["G"]
    r = np.random.default_rng(0)
    rows = r.integers(0, k, 64)
    cols = r.integers(0, n, 64)
    got = _np(G[torch.tensor(rows, device="cuda"), torch.tensor(cols, device="cuda")])
    want = np.array([rng.gaussian_block(seed, n, [a], [b], "bf16")[0, 0] for a, b in zip(rows, cols)])
    assert np.array_equal(got, want)
    del G
    sk.close()


# ---------------------------------------------------------------------------
# RHSketch (Algorithm 1)
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
@pytest.mark.parametrize("n,m,c,k", [(1000, 8, 8, 64), (4097, 0, 3, 100), (20000, 33, 40, 128), (9000, 5, 1, 16)])
def test_sketch_apply_f64(gpu_lib, kind, n, m, c, k):
    from paper_2405_10923_gb300 import torch_api as ta

    X = ri.gaussian(n, c, 5)
    if kind == "srht":
        sk, osk = ta.Sketch(n, k, gpu_lib.SRHT, 3), sketch.SRHTSketch(n, k, 3)
    else:
        sk, osk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, 3), sketch.GaussianSketch(n, k, 3)
    Z = _np(sk.apply(_dev(X), m))
    Zo = sketch.rh_sketch(X, m, osk)
    assert np.array_equal(Z[:m], Zo[:m])
    assert np.max(np.abs(Z - Zo)) <= 1e-13 * np.abs(Zo).max()
    sk.close()


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("n,m,c,k", [(200, 3, 2, 16), (300, 0, 3, 40), (700, 5, 2, 64), (2000, 7, 1, 64),
                                     (3000, 2, 4, 128), (6000, 9, 2, 256), ((1 << 20) + 5, 16, 2, 512)])
def test_srht_every_segment_length(gpu_lib, dt, n, m, c, k):
    """The SRHT's transform runs per segment of N2 = min(N, 8192) entries: in
    shared memory one level at a time below 512 entries, by the register /
    warp-shuffle / one-transpose kernel from 512 to 8192.  Every length against
    the oracle's Sylvester transform (float64 to 1e-13; float32 within the
    float32 bound gamma_{log2 N + 5} of the SRHT lemma)."""
    from paper_2405_10923_gb300 import torch_api as ta

    X = ri.gaussian(n, c, 8)
    if dt == "f32":
        X = X.astype(np.float32).astype(np.float64)
    sk, osk = ta.Sketch(n, k, gpu_lib.SRHT, 9), sketch.SRHTSketch(n, k, 9)
    Z = _np(sk.apply(_dev(X, torch.float64 if dt == "f64" else torch.float32), m))
    Zo = sketch.rh_sketch(X, m, osk)
    assert np.array_equal(Z[:m], Zo[:m])
    if dt == "f64":
        assert np.max(np.abs(Z - Zo)) <= 1e-13 * np.abs(Zo).max()
    else:
        lg = int(np.ceil(np.log2(n)))
        gamma = (lg + 5) * 2.0**-24 / (1 - (lg + 5) * 2.0**-24)
        colnorm = np.linalg.norm(X[m:], axis=0)
        assert (np.abs(Z[m:] - Zo[m:]).max(axis=0) <= gamma * np.sqrt(2.0**lg / k) * colnorm).all()
    sk.close()


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
def test_sketch_apply_f32(gpu_lib, kind):
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, c, k = 50000, 16, 16, 128
    X = ri.gaussian(n, c, 6).astype(np.float32).astype(np.float64)
    if kind == "srht":
        sk, osk = ta.Sketch(n, k, gpu_lib.SRHT, 4), sketch.SRHTSketch(n, k, 4)
    else:
        sk, osk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, 4, gpu_lib.F32), sketch.GaussianSketch(n, k, 4, "f32")
    Z = _np(sk.apply(_dev(X, torch.float32), m))
    Zo = sketch.rh_sketch(X, m, osk)
    # float32 accumulation: about log2(N) (SRHT) or sqrt(chunk) (Gaussian) roundings
    assert np.max(np.abs(Z - Zo)) <= 2e-5 * np.abs(Zo).max()
    sk.close()


# ---------------------------------------------------------------------------
# factorisations
# ---------------------------------------------------------------------------


def _check_factors(out, ref, tol):
    U, S, T, R = ref[:4]
    scale = np.abs(R).max()
    assert np.max(np.abs(_np(out["R"]) - R)) <= tol * scale
    assert np.max(np.abs(_np(out["S"]) - S)) <= tol * max(1, np.abs(S).max())
    assert np.max(np.abs(_np(out["T"]) - T)) <= tol * max(1, np.abs(T).max())
    if out["U"] is not None:
        assert np.max(np.abs(_np(out["U"]) - U)) <= tol * max(1, np.abs(U).max())


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
@pytest.mark.parametrize("n,m,k", [(1000, 8, 32), (4096, 32, 128), (10007, 20, 64)])
def test_rec_rhqr_f64_matches_oracle(gpu_lib, kind, n, m, k):
    from paper_2405_10923_gb300 import torch_api as ta

    W = ri.gaussian(n, m, 10)
    if kind == "srht":
        sk, osk = ta.Sketch(n, k, gpu_lib.SRHT, 12), sketch.SRHTSketch(n, k, 12)
    else:
        sk, osk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, 12), sketch.GaussianSketch(n, k, 12)
    out = ta.factor(sk, _dev(W), alg=gpu_lib.ALG_REC, want_U=True)
    torch.cuda.synchronize()
    assert ta.info(out)["status"] == 0
    ref = rhqr.rec_rhqr(W, osk)
    _check_factors(out, ref, 1e-11)
    Q = _np(out["Q"])
    Qo = rhqr.form_q(ref[0], ref[2])
    assert np.max(np.abs(Q - Qo)) <= 1e-11
    assert metrics.sketch_orthogonality(Q, osk) <= 1e-12
    assert metrics.residual(W, Q, _np(out["R"])) <= 1e-12
    # Q only (no U): Q = W R^{-1} by the row solve
    out2 = ta.factor(sk, _dev(W), alg=gpu_lib.ALG_REC, want_U=False)
    assert np.max(np.abs(_np(out2["Q"]) - Qo)) <= 1e-11
    sk.close()


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
@pytest.mark.parametrize("n,m,k", [(4096, 32, 128), (3001, 7, 40), (20000, 48, 96)])
def test_left_rhqr_f64_matches_oracle(gpu_lib, kind, n, m, k):
    from paper_2405_10923_gb300 import torch_api as ta

    W = ri.gaussian(n, m, 20)
    if kind == "srht":
        sk, osk = ta.Sketch(n, k, gpu_lib.SRHT, 21), sketch.SRHTSketch(n, k, 21)
    else:
        sk, osk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, 21), sketch.GaussianSketch(n, k, 21)
    out = ta.factor(sk, _dev(W), alg=gpu_lib.ALG_LEFT)
    torch.cuda.synchronize()
    assert ta.info(out)["status"] == 0
    ref = rhqr.rhqr_left(W, osk)
    _check_factors(out, ref, 1e-11)
    Qo = rhqr.form_q(ref[0], ref[2])
    assert np.max(np.abs(_np(out["Q"]) - Qo)) <= 1e-11
    sk.close()


def test_left_rhqr_norm_scaling(gpu_lib):
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 2000, 6, 24
    W = ri.gaussian(n, m, 22)
    sk, osk = ta.Sketch(n, k, gpu_lib.SRHT, 23), sketch.SRHTSketch(n, k, 23)
    out = ta.factor(sk, _dev(W), alg=gpu_lib.ALG_LEFT, scaling=1)
    ref = rhqr.rhqr_left(W, osk, scaling="norm")
    _check_factors(out, ref, 1e-11)
    sk.close()


@pytest.mark.parametrize("cond", [1e4, 1e10])
def test_left_rhqr_f32_invariants(gpu_lib, cond):
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 1 << 16, 32, 128
    W = ri.spectrum(n, m, cond, 30).astype(np.float32).astype(np.float64)
    sk, osk = ta.Sketch(n, k, gpu_lib.SRHT, 31), sketch.SRHTSketch(n, k, 31)
    out = ta.factor(sk, _dev(W, torch.float32), alg=gpu_lib.ALG_LEFT)
    torch.cuda.synchronize()
    assert ta.info(out)["status"] == 0
    Q = _np(out["Q"])
    assert metrics.sketch_orthogonality(Q, osk) <= 1e-5
    assert metrics.residual(W, Q, _np(out["R"])) <= 1e-5
    sk.close()


def test_rec_refinement_f64_high_condition(gpu_lib):
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 1 << 15, 16, 64
    W = ri.spectrum(n, m, 1e12, 40)
    sk, osk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, 41), sketch.GaussianSketch(n, k, 41)
    out = ta.factor(sk, _dev(W), alg=gpu_lib.ALG_REC, passes=2)
    torch.cuda.synchronize()
    assert ta.info(out)["passes_done"] == 2
    Qo, Ro, *_ = rhqr.rec_rhqr_refined(W, osk, passes=2)
    Q = _np(out["Q"])
    assert metrics.sketch_orthogonality(Q, osk) <= 1e-12
    assert metrics.residual(W, Q, _np(out["R"])) <= 1e-12
    sk.close()


def test_reconstruct_matches_oracle(gpu_lib):
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 5000, 12, 48
    W = ri.gaussian(n, m, 50)
    osk = sketch.GaussianSketch(n, k, 51)
    sk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, 51)
    Z = sketch.rh_sketch(W, m, osk)
    S, T, R = rhqr.householder_qr(Z)
    Ud, Qd = ta.reconstruct(sk, _dev(S), _dev(T), _dev(R), _dev(Z), _dev(W))
    U, *_ = rhqr.rec_rhqr(W, osk)
    assert np.max(np.abs(_np(Ud) - U)) <= 1e-11
    assert np.max(np.abs(_np(Qd) - rhqr.form_q(U, T))) <= 1e-11
    sk.close()


def test_breakdown_is_reported(gpu_lib):
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 1000, 4, 16
    W = ri.gaussian(n, m, 60)
    W[:, 2] = 0.0  # a zero column: rho = 0 at column 2
    sk = ta.Sketch(n, k, gpu_lib.SRHT, 61)
    for alg in (gpu_lib.ALG_LEFT, gpu_lib.ALG_REC):
        out = ta.factor(sk, _dev(W), alg=alg)
        torch.cuda.synchronize()
        info = ta.info(out)
        assert info["status"] == 4 and info["column"] == 2, info
    sk.close()


def test_nonfinite_is_reported(gpu_lib):
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 1000, 4, 16
    W = ri.gaussian(n, m, 62)
    W[500, 1] = np.nan
    sk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, 63)
    out = ta.factor(sk, _dev(W), alg=gpu_lib.ALG_REC)
    torch.cuda.synchronize()
    assert ta.info(out)["status"] == 5
    sk.close()
