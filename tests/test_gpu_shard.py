"""Row-partitioned sketching (rhqr_sketch_apply_rows): a matrix split by rows,
each holder sketching its own rows with the library's kernels, one sum of the
(k+m) x c results giving Z = Psi_m X (Algorithm 1's single synchronization).

The shards' sum is compared with the whole-matrix sketch of the same library
(float64: 1e-13 relative, the two only differ in summation order) and with
the oracle's RHSketch; a two-process run over gloo (ranks on the same GPU,
no kernel waits on another rank: the all-reduce runs on host copies) shows
the distributed use end to end."""

import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

import rhqr_inputs as ri  # noqa: E402
from oracle import sketch  # noqa: E402


def _sk(gpu_lib, kind, n, k, seed, dt=None):
    from paper_2405_10923_gb300 import torch_api as ta

    if kind == "srht":
        return ta.Sketch(n, k, gpu_lib.SRHT, seed), sketch.SRHTSketch(n, k, seed)
    return ta.Sketch(n, k, gpu_lib.GAUSSIAN, seed, dt or gpu_lib.F64), sketch.GaussianSketch(n, k, seed)


def _bounds(n, parts, align):
    cuts = [0]
    for p in range(1, parts):
        cuts.append((n * p // parts) // align * align)
    cuts.append(n)
    return cuts


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
@pytest.mark.parametrize("n,m,c,k,parts", [(20000, 8, 5, 64, 2), (40000, 33, 3, 128, 3), (9000, 0, 2, 32, 4),
                                           (100000, 12, 4, 256, 5)])
def test_shards_sum_to_the_sketch(gpu_lib, kind, n, m, c, k, parts):
    import paper_2405_10923_gb300 as rh

    X = ri.gaussian(n, c, 30)
    sk, osk = _sk(gpu_lib, kind, n, k, 31)
    align = sk.N if kind == "srht" and sk.N <= 8192 else (8192 if kind == "srht" else 1)
    cuts = _bounds(n, parts, align)
    Xd = rh.colmajor(torch.tensor(X, device="cuda"))
    Zfull = sk.apply(Xd, m).cpu().numpy()
    Zsum = np.zeros_like(Zfull)
    for a, b in zip(cuts[:-1], cuts[1:]):
        if b <= a:
            continue
        Xl = rh.colmajor(torch.tensor(X[a:b], device="cuda"))
        Zsum += sk.apply_rows(Xl, m, a).cpu().numpy()
    assert np.array_equal(Zsum[:m], X[:m])
    assert np.max(np.abs(Zsum - Zfull)) <= 1e-13 * np.abs(Zfull).max()
    Zo = sketch.rh_sketch(X, m, osk)
    assert np.max(np.abs(Zsum - Zo)) <= 1e-13 * np.abs(Zo).max()
    sk.close()


def test_srht_shards_must_start_on_a_segment(gpu_lib):
    import paper_2405_10923_gb300 as rh

    n, k = 1 << 15, 64
    sk, _ = _sk(gpu_lib, "srht", n, k, 32)
    Xl = rh.colmajor(torch.zeros((1000, 2), dtype=torch.float64, device="cuda"))
    with pytest.raises(gpu_lib.RHQRError) as e:
        sk.apply_rows(Xl, 4, 100)
    assert e.value.code == 1
    sk.close()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, m, c, k, out_path):
    import torch.distributed as dist

    import paper_2405_10923_gb300 as rh
    from paper_2405_10923_gb300 import torch_api as ta

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    rh.load()
    X = ri.gaussian(n, c, 33)  # every rank draws the same matrix and keeps its rows
    sk = ta.Sketch(n, k, rh.SRHT, 34)
    seg = min(sk.N, 8192)
    cuts = _bounds(n, world, seg)
    a, b = cuts[rank], cuts[rank + 1]
    Z = sk.apply_rows(rh.colmajor(torch.tensor(X[a:b], device="cuda")), m, a).cpu()
    dist.all_reduce(Z, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(out_path, Z.numpy())
    sk.close()
    dist.destroy_process_group()


def test_two_ranks_over_gloo(gpu_lib, tmp_path):
    import torch.multiprocessing as mp

    n, m, c, k = 50000, 10, 3, 128
    out = str(tmp_path / "z.npy")
    mp.spawn(_rank_main, args=(2, _free_port(), n, m, c, k, out), nprocs=2, join=True)
    Z = np.load(out)
    X = ri.gaussian(n, c, 33)
    Zo = sketch.rh_sketch(X, m, sketch.SRHTSketch(n, k, 34))
    assert np.max(np.abs(Z - Zo)) <= 1e-13 * np.abs(Zo).max()
