"""RHQR-Arnoldi step (Algorithm 7) on the GPU vs the oracle, through the C ABI.

The test plays the caller: it applies the operator to the basis vector the
library returns and feeds A q_j back.  float64 basis: h_j, q_j and the compact
factors (U, S, T) agree with the oracle to 1e-11 (relative); the Arnoldi
relation A Q_m = Q_{m+1} H and the orthonormality of Psi Q_{m+1} hold to
1e-12.  float32 basis: both invariants <= 1e-5."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import rhqr_inputs as ri  # noqa: E402
from oracle import rhqr, sketch  # noqa: E402


def _run(gpu_lib, kind, n, k, mmax, A, dtype, seed=3, scaling=0):
    from paper_2405_10923_gb300 import torch_api as ta

    if kind == "srht":
        sk, osk = ta.Sketch(n, k, gpu_lib.SRHT, seed), sketch.SRHTSketch(n, k, seed)
    else:
        sk, osk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, seed), sketch.GaussianSketch(n, k, seed)
    b = np.random.default_rng(seed + 1).standard_normal(n)
    if dtype == torch.float32:
        b = b.astype(np.float32).astype(np.float64)
    arn = ta.Arnoldi(sk, n, mmax, dtype=dtype, scaling=scaling)
    h0, q = arn.begin(torch.tensor(b, dtype=dtype, device="cuda"))
    Q, H = [q.double().cpu().numpy()], []
    for _ in range(mmax):
        w = A(Q[-1])
        if dtype == torch.float32:
            w = w.astype(np.float32).astype(np.float64)
        h, q = arn.step(torch.tensor(w, dtype=dtype, device="cuda"))
        H.append(h.cpu().numpy())
        Q.append(q.double().cpu().numpy())
    torch.cuda.synchronize()
    info = gpu_lib.read_info(arn.info)
    U, S, T, cnt = arn.export()
    out = dict(h0=h0.cpu().numpy(), H=np.stack(H, axis=1), Q=np.stack(Q, axis=1), U=U.double().cpu().numpy(),
               S=S.cpu().numpy(), T=T.cpu().numpy(), count=cnt, info=info)
    arn.close()
    sk.close()
    return out, osk, b


def _dense(n, seed):
    M = np.random.default_rng(seed).standard_normal((n, n)) / np.sqrt(n) + 2 * np.eye(n)
    return M, (lambda x: M @ x)


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
def test_arnoldi_f64_matches_oracle(gpu_lib, kind):
    n, k, mmax = 1600, 64, 12
    Amat, Aop = _dense(n, 5)
    out, osk, b = _run(gpu_lib, kind, n, k, mmax, Aop, torch.float64)
    assert out["info"]["status"] == 0 and out["count"] == mmax + 1
    H, Qo, h0o, arn = rhqr.rhqr_arnoldi(Aop, b, np.zeros(n), osk, mmax)
    assert np.max(np.abs(out["h0"] - h0o)) <= 1e-11 * np.abs(h0o).max()
    assert np.max(np.abs(out["H"] - H)) <= 1e-11 * np.abs(H).max()
    assert np.max(np.abs(out["Q"] - Qo)) <= 1e-11
    assert np.max(np.abs(out["U"] - arn.U)) <= 1e-11 * max(1, np.abs(arn.U).max())
    assert np.max(np.abs(out["S"] - arn.S)) <= 1e-11 * max(1, np.abs(arn.S).max())
    assert np.max(np.abs(out["T"] - arn.T)) <= 1e-11 * max(1, np.abs(arn.T).max())
    Q = out["Q"]
    assert np.max(np.abs(Amat @ Q[:, :mmax] - Q @ out["H"])) <= 1e-12 * np.abs(Amat).max() * 10
    PQ = sketch.rh_sketch(Q, mmax + 1, osk)
    assert np.max(np.abs(PQ.T @ PQ - np.eye(mmax + 1))) <= 1e-12


def test_arnoldi_stencil_f32(gpu_lib):
    g = 64
    n, k, mmax = g * g, 96, 20
    Aop = lambda x: ri.stencil_apply(x.copy(), g)  # noqa: E731
    out, osk, b = _run(gpu_lib, "srht", n, k, mmax, Aop, torch.float32)
    assert out["info"]["status"] == 0
    Q, H = out["Q"], out["H"]
    AQ = np.stack([Aop(Q[:, j]) for j in range(mmax)], axis=1)
    assert np.linalg.norm(AQ - Q @ H) / np.linalg.norm(AQ) <= 1e-5
    PQ = sketch.rh_sketch(Q, mmax + 1, osk)
    assert np.max(np.abs(PQ.T @ PQ - np.eye(mmax + 1))) <= 1e-5


def test_arnoldi_norm_scaling_and_breakdown(gpu_lib):
    from paper_2405_10923_gb300 import torch_api as ta

    n, k, mmax = 1000, 40, 6
    Amat, Aop = _dense(n, 7)
    out, osk, b = _run(gpu_lib, "srht", n, k, mmax, Aop, torch.float64, scaling=1)
    H, Qo, h0o, arn = rhqr.rhqr_arnoldi(Aop, b, np.zeros(n), osk, mmax, scaling="norm")
    assert np.max(np.abs(out["H"] - H)) <= 1e-11 * np.abs(H).max()
    assert np.max(np.abs(out["Q"] - Qo)) <= 1e-11
    # r0 = 0: rho = 0 at the first reflector
    sk = ta.Sketch(n, k, gpu_lib.SRHT, 9)
    arnd = ta.Arnoldi(sk, n, mmax)
    arnd.begin(torch.zeros(n, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    info = gpu_lib.read_info(arnd.info)
    assert info["status"] == 4 and info["column"] == 0
    arnd.close()
    sk.close()
