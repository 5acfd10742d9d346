"""Host-memory factorisation stream (rhqr_pipeline_*): every submission gives,
bit for bit, what rhqr_factor gives on the same matrix held on the device
(the pipeline adds transfers and event ordering, no arithmetic), and the
float64 left-looking results also match the oracle."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import rhqr_inputs as ri  # noqa: E402
from oracle import rhqr, sketch  # noqa: E402


def _host_colmajor(a, dtype, ld=None):
    rows, cols = a.shape
    ld = rows if ld is None else ld
    buf = torch.zeros((cols, ld), dtype=dtype, pin_memory=True)
    out = buf.t()[:rows]
    out.copy_(torch.as_tensor(a, dtype=dtype))
    return out


def _run(gpu_lib, sk, Ws, opts, dtype, depth, ldw_pad=0):
    from paper_2405_10923_gb300 import torch_api as ta

    n, m = Ws[0].shape
    pipe = ta.Pipeline(sk, n, m, dtype=dtype, opts=opts, depth=depth)
    Wh = [_host_colmajor(W, dtype, n + ldw_pad) for W in Ws]
    Qh = [ta.Pipeline.host_colmajor(n, m, dtype) for _ in Ws]
    Rh = [ta.Pipeline.host_colmajor(m, m, torch.float64) for _ in Ws]
    Sh = [ta.Pipeline.host_colmajor(sk.k + m, m, torch.float64) for _ in Ws]
    Th = [ta.Pipeline.host_colmajor(m, m, torch.float64) for _ in Ws]
    info = [torch.zeros(4, dtype=torch.int32).pin_memory() for _ in Ws]
    for i in range(len(Ws)):
        pipe.submit(Wh[i], Qh[i], Rh[i], Sh[i], Th[i], info[i])
    pipe.wait()
    pipe.close()
    return Qh, Rh, Sh, Th, info


def _direct(gpu_lib, sk, W, opts, dtype):
    from paper_2405_10923_gb300 import torch_api as ta

    n = W.shape[0]
    Wd = gpu_lib.colmajor(torch.as_tensor(W, dtype=dtype, device="cuda"), ld=(n + 31) // 32 * 32)
    out = ta.factor(sk, Wd, opts=opts)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_pipeline_rec_f32_bitwise_equal_to_factor(gpu_lib, depth):
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = (1 << 16) + 96, 64, 256  # ragged against 128-row tiles
    sk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, 31, gpu_lib.BF16)
    opts = ta.make_opts(alg=gpu_lib.ALG_REC, passes=3)
    Ws = [ri.spectrum(n, m, 10.0 ** (2 + 3 * i), 40 + i) for i in range(4)]
    Qh, Rh, Sh, Th, info = _run(gpu_lib, sk, Ws, opts, torch.float32, depth, ldw_pad=5)
    for i, W in enumerate(Ws):
        ref = _direct(gpu_lib, sk, W, opts, torch.float32)
        assert info[i].tolist() == ref["info"].cpu().tolist(), i
        assert int(info[i][0]) == 0
        assert torch.equal(Qh[i], ref["Q"].cpu()), i
        assert torch.equal(Rh[i], ref["R"].cpu()), i
        assert torch.equal(Sh[i], ref["S"].cpu()), i
        assert torch.equal(Th[i], ref["T"].cpu()), i
    sk.close()


def test_pipeline_left_f64_matches_factor_and_oracle(gpu_lib):
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 3000, 12, 48
    sk = ta.Sketch(n, k, gpu_lib.SRHT, 77)
    opts = ta.make_opts(alg=gpu_lib.ALG_LEFT)
    Ws = [ri.gaussian(n, m, 900 + i) for i in range(3)]
    Qh, Rh, Sh, Th, info = _run(gpu_lib, sk, Ws, opts, torch.float64, 2)
    osk = sketch.SRHTSketch(n, k, 77)
    for i, W in enumerate(Ws):
        ref = _direct(gpu_lib, sk, W, opts, torch.float64)
        assert torch.equal(Qh[i], ref["Q"].cpu()), i
        assert torch.equal(Rh[i], ref["R"].cpu()), i
        U, S, T, R = rhqr.rhqr_left(W, osk)
        scale = np.abs(R).max()
        assert np.max(np.abs(Rh[i].numpy() - R)) <= 1e-10 * scale, i
        assert np.max(np.abs(Qh[i].numpy() - rhqr.form_q(U, T))) <= 1e-10, i
    sk.close()


def test_pipeline_reports_breakdown_in_host_info(gpu_lib):
    from paper_2405_10923_gb300 import torch_api as ta

    n, m, k = 4096, 8, 32
    sk = ta.Sketch(n, k, gpu_lib.SRHT, 5)
    W = ri.gaussian(n, m, 3)
    W[:, 5] = 0.0  # a zero column: rho = 0 at column 5
    opts = ta.make_opts(alg=gpu_lib.ALG_REC)
    _, _, _, _, info = _run(gpu_lib, sk, [W, ri.gaussian(n, m, 4)], opts, torch.float64, 2)
    assert int(info[0][0]) == 4 and int(info[0][1]) == 5  # RHQR_EBREAKDOWN at column 5
    assert int(info[1][0]) == 0
    sk.close()
