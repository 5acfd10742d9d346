"""Batched recRHQR (Algorithm 6 with refinement passes) over ragged problems,
through the C ABI, against the FP64 oracle problem by problem.

float64 data: factors agree with the oracle to 1e-10 relative and every
problem meets ||I - (Psi Q)^t Psi Q||_2, ||W - QR||_F/||W||_F <= 1e-12.
float32 data (three passes, Gaussian and cond 1e8 spectra mixed): both
measures <= 1e-5.  Launch-shape choices of the tuner and CUDA-graph replay
change no arithmetic, so their results are compared bit for bit."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import rhqr_inputs as ri  # noqa: E402
from oracle import metrics, rhqr, sketch  # noqa: E402


def _np(t):
    return t.detach().double().cpu().numpy()


def _batch(gpu_lib, Ws, ks, seeds, dtype, **kw):
    from paper_2405_10923_gb300 import torch_api as ta

    sks = [ta.Sketch(W.shape[0], k, gpu_lib.SRHT, s) for W, k, s in zip(Ws, ks, seeds)]
    Wd = [gpu_lib.colmajor(torch.tensor(W, dtype=dtype, device="cuda")) for W in Ws]
    return ta.Batch(sks, Wd, **kw), sks


def _ragged(count, seed, n_lo=700, n_hi=9000, ms=(3, 16, 33, 64)):
    n, m = ri.ragged_batch(count, n_lo, n_hi, ms, seed)
    return [int(x) for x in n], [int(x) for x in m]


def test_batched_f64_matches_oracle(gpu_lib):
    ns, ms = _ragged(7, 1)
    ns[0], ms[0] = 600, 128  # the largest m, with k = 4m = 512 < n
    Ws = [ri.gaussian(n, m, 100 + i) for i, (n, m) in enumerate(zip(ns, ms))]
    ks = [4 * m for m in ms]
    seeds = [200 + i for i in range(len(Ws))]
    b, sks = _batch(gpu_lib, Ws, ks, seeds, torch.float64, passes=1)
    b.run()
    torch.cuda.synchronize()
    for i, (W, k, s) in enumerate(zip(Ws, ks, seeds)):
        assert b.infos()[i]["status"] == 0 and b.infos()[i]["passes_done"] == 1
        osk = sketch.SRHTSketch(W.shape[0], k, s)
        U, S, T, R, _M = rhqr.rec_rhqr(W, osk)
        scale = np.abs(R).max()
        assert np.max(np.abs(_np(b.R[i]) - R)) <= 1e-10 * scale, i
        assert np.max(np.abs(_np(b.S[i]) - S)) <= 1e-10 * max(1, np.abs(S).max()), i
        assert np.max(np.abs(_np(b.T[i]) - T)) <= 1e-10 * max(1, np.abs(T).max()), i
        Q = _np(b.Q[i])
        assert np.max(np.abs(Q - rhqr.form_q(U, T))) <= 1e-10, i
        assert metrics.sketch_orthogonality(Q, osk) <= 1e-12, i
        assert metrics.residual(W, Q, _np(b.R[i])) <= 1e-12, i
    b.close()


def test_batched_f64_refined_matches_oracle(gpu_lib):
    ns, ms = _ragged(4, 2)
    Ws = [ri.spectrum(n, m, 1e12, 300 + i) for i, (n, m) in enumerate(zip(ns, ms))]
    ks = [4 * m for m in ms]
    seeds = [400 + i for i in range(len(Ws))]
    b, _ = _batch(gpu_lib, Ws, ks, seeds, torch.float64, passes=2)
    b.run()
    torch.cuda.synchronize()
    for i, (W, k, s) in enumerate(zip(Ws, ks, seeds)):
        assert b.infos()[i]["passes_done"] == 2
        osk = sketch.SRHTSketch(W.shape[0], k, s)
        Q = _np(b.Q[i])
        assert metrics.sketch_orthogonality(Q, osk) <= 1e-12, i
        assert metrics.residual(W, Q, _np(b.R[i])) <= 1e-12, i
    b.close()


def test_batched_f32_three_passes_meets_bound(gpu_lib):
    ns, ms = _ragged(8, 3, n_lo=2000, n_hi=40000, ms=(16, 32, 64, 128))
    Ws = []
    for i, (n, m) in enumerate(zip(ns, ms)):
        W = ri.gaussian(n, m, 500 + i) if i % 2 == 0 else ri.spectrum(n, m, 1e8, 500 + i)
        Ws.append(ri.to_dtype(W, "f32").astype(np.float64))
    ks = [4 * m for m in ms]
    seeds = [600 + i for i in range(len(Ws))]
    b, _ = _batch(gpu_lib, Ws, ks, seeds, torch.float32, passes=3)
    b.run()
    torch.cuda.synchronize()
    for i, (W, k, s) in enumerate(zip(Ws, ks, seeds)):
        assert b.infos()[i]["status"] == 0, (i, b.infos()[i])
        osk = sketch.SRHTSketch(W.shape[0], k, s)
        Q = _np(b.Q[i])
        assert metrics.sketch_orthogonality(Q, osk) <= 1e-5, i
        assert metrics.residual(W, Q, _np(b.R[i])) <= 1e-5, i
        if i % 2 == 0:  # well conditioned: R is determined to working accuracy
            Ro = rhqr.rec_rhqr_refined(W, osk, passes=3)[1]
            assert np.max(np.abs(_np(b.R[i]) - Ro)) <= 1e-4 * np.abs(Ro).max(), i
    b.close()


def test_batched_graph_replay_and_tuning_are_bit_identical(gpu_lib, tmp_path):
    ns, ms = _ragged(9, 4, ms=(16, 32, 64, 128))
    ns = [max(n, 4 * m + 1) for n, m in zip(ns, ms)]
    Ws = [ri.gaussian(n, m, 700 + i) for i, (n, m) in enumerate(zip(ns, ms))]
    b, _ = _batch(gpu_lib, Ws, [4 * m for m in ms], [800 + i for i in range(len(Ws))], torch.float32, passes=2)
    b.run()
    torch.cuda.synchronize()
    Q0 = [q.clone() for q in b.Q]
    R0 = [r.clone() for r in b.R]
    cache = str(tmp_path / "tune.json")
    choice = b.tune(reps=2, cache=cache)
    assert choice[0] in (128, 256, 512, 1024) and choice[1] in (32, 64, 128)
    assert b.tune(cache=cache) == tuple(choice)  # served from the cache
    for c in [(128, 32, 0), (1024, 128, 152 * 4), tuple(choice)]:
        gpu_lib.rhqr_batch_set_tuning(b.handle, c)
        for q in b.Q:
            q.zero_()
        b.run()
        torch.cuda.synchronize()
        for i in range(len(Ws)):
            assert torch.equal(b.Q[i], Q0[i]) and torch.equal(b.R[i], R0[i]), (c, i)
    g = b.capture()
    for q in b.Q:
        q.zero_()
    g.replay()
    torch.cuda.synchronize()
    for i in range(len(Ws)):
        assert torch.equal(b.Q[i], Q0[i]) and torch.equal(b.R[i], R0[i]), i
    with pytest.raises(gpu_lib.RHQRError):
        gpu_lib.rhqr_batch_set_tuning(b.handle, (100, 64, 0))
    b.close()


def test_batched_breakdown_is_local(gpu_lib):
    Ws = [ri.gaussian(1000, 4, 900), ri.gaussian(1500, 6, 901), ri.gaussian(800, 5, 902)]
    Ws[1][:, 2] = 0.0  # rho = 0 at column 2 of problem 1 only
    b, _ = _batch(gpu_lib, Ws, [16, 24, 20], [910, 911, 912], torch.float64, passes=1)
    b.run()
    torch.cuda.synchronize()
    infos = b.infos()
    assert infos[1]["status"] == 4 and infos[1]["column"] == 2, infos
    for i in (0, 2):
        assert infos[i]["status"] == 0
        osk = sketch.SRHTSketch(Ws[i].shape[0], [16, 24, 20][i], 910 + i)
        assert metrics.sketch_orthogonality(_np(b.Q[i]), osk) <= 1e-12
    b.close()


def test_batched_argument_errors(gpu_lib):
    from paper_2405_10923_gb300 import torch_api as ta

    sk = ta.Sketch(1000, 16, gpu_lib.SRHT, 1)
    gk = ta.Sketch(1000, 16, gpu_lib.GAUSSIAN, 1)
    W = gpu_lib.colmajor(torch.zeros((1000, 4), dtype=torch.float64, device="cuda"))
    with pytest.raises(gpu_lib.RHQRError):  # Gaussian sketch
        ta.Batch([gk], [W])
    with pytest.raises(gpu_lib.RHQRError):  # m > k
        ta.Batch([sk], [gpu_lib.colmajor(torch.zeros((1000, 20), dtype=torch.float64, device="cuda"))])
    with pytest.raises(gpu_lib.RHQRError):  # float16 data
        ta.Batch([sk], [gpu_lib.colmajor(torch.zeros((1000, 4), dtype=torch.float16, device="cuda"))])
    b = ta.Batch([sk], [W])
    with pytest.raises(gpu_lib.RHQRError):  # workspace too small
        gpu_lib.rhqr_factor_batched(b.handle, b.ws, b.ws_bytes - 1, b.info)
    b.close()
    sk.close()
    gk.close()


def test_batched_full_size_sampled(gpu_lib):
    """The full ragged workload (512 float32 problems, n_i log-uniform in
    [16384, 262144], m_i in {16, 32, 64, 128}, k_i = 4 m_i, half Gaussian and
    half cond 1e8 spectra, three passes) in the launch configuration the tuner
    picks, replayed from a CUDA graph; sampled problems are checked with the
    oracle's sketch, every problem's status and passes on the device."""
    from paper_2405_10923_gb300 import torch_api as ta

    Ws, ns, ms = ri.device_ragged_batch(512, 16384, 262144, (16, 32, 64, 128), 1e8, 4, torch.float32)
    sks = [ta.Sketch(n, 4 * m, gpu_lib.SRHT, 7000 + i) for i, (n, m) in enumerate(zip(ns, ms))]
    b = ta.Batch(sks, Ws, passes=3)
    b.tune(reps=1)
    g = b.capture()
    for q in b.Q:
        q.zero_()
    g.replay()
    torch.cuda.synchronize()
    infos = b.infos()
    assert all(x["status"] == 0 and x["passes_done"] == 3 for x in infos)
    big = max(range(512), key=lambda i: ns[i] * ms[i])
    for i in sorted({0, 1, 255, 510, 511, big}):
        W = _np(Ws[i])
        osk = sketch.SRHTSketch(ns[i], 4 * ms[i], 7000 + i)
        Q = _np(b.Q[i])
        assert metrics.sketch_orthogonality(Q, osk) <= 1e-5, i
        assert metrics.residual(W, Q, _np(b.R[i])) <= 1e-5, i
    b.close()
