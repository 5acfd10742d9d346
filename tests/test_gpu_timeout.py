"""Bounded device-side waits: a wait that runs out is reported, not hung on.

Every mbarrier wait of the tensor-core kernels (the Gaussian sketch and both
row solves) gives up after rhqr_opts.wait_budget polls.  With a budget of one
poll the waits run out long before the copies and MMAs they wait for arrive:
the call must come back with RHQR_ETIMEOUT in its rhqr_info, and the device
must stay usable -- the blocks that stopped let their copies and MMAs in
flight finish and release their tensor memory, so the next call (default
budget) runs and gives, bit for bit, the result of a call made before.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import rhqr_inputs as ri  # noqa: E402

ETIMEOUT = 6


@pytest.mark.parametrize("solve", [0, 1])
@pytest.mark.parametrize("kind,m", [("gaussian_bf16", 128), ("srht", 128), ("gaussian_bf16", 256)])
def test_tiny_wait_budget_times_out_and_recovers(gpu_lib, kind, m, solve):
    """m = 256 sketches two column tiles of X on CTA pairs (cta_group::2)."""
    import paper_2405_10923_gb300 as rh
    from paper_2405_10923_gb300 import torch_api as ta

    n, k = 1 << 18, 512
    W = rh.colmajor(torch.tensor(ri.gaussian(n, m, 50), dtype=torch.float32, device="cuda"))
    if kind == "srht":
        sk = ta.Sketch(n, k, gpu_lib.SRHT, 51)
    else:
        sk = ta.Sketch(n, k, gpu_lib.GAUSSIAN, 51, gpu_lib.BF16)
    ref = ta.factor(sk, W, alg=gpu_lib.ALG_REC, passes=2, solve=solve)
    torch.cuda.synchronize()
    assert ta.info(ref)["status"] == 0
    Q0, R0 = ref["Q"].clone(), ref["R"].clone()

    bad = ta.factor(sk, W, alg=gpu_lib.ALG_REC, passes=2, solve=solve, wait_budget=1, ws=ref["ws"])
    torch.cuda.synchronize()
    assert ta.info(bad)["status"] == ETIMEOUT

    again = ta.factor(sk, W, alg=gpu_lib.ALG_REC, passes=2, solve=solve, ws=ref["ws"])
    torch.cuda.synchronize()
    assert ta.info(again)["status"] == 0
    assert torch.equal(again["Q"], Q0) and torch.equal(again["R"], R0)
    assert np.isfinite(again["Q"].cpu().numpy()).all()
    sk.close()
