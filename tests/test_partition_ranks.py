"""The row-partitioned sketch (the multi-GPU layout of the path: W split by rows,
one sum over ranks of the per-shard sketches, everything after it replicated)
on two gloo ranks on CPU: the sum of the shards' partial sketches equals the
oracle's sketch of the whole matrix, for the Gaussian operator (columns of
Omega_full per shard, Section 2.3) and for the SRHT (each shard transforms its
half of the zero-padded rows; the Sylvester Hadamard matrix of size N is
H_2 (x) H_{N/2}, so the shard's transform enters the sum with the entry of H_2
that its block meets in the sampled row)."""

import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import rhqr_inputs as ri  # noqa: E402
from oracle import sketch  # noqa: E402

N_ROWS, M, K = 3000, 6, 40


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shard_sketch(rank: int, world: int, kind: str):
    W = ri.gaussian(N_ROWS, M, 11)
    if kind == "gaussian":
        sk = sketch.GaussianSketch(N_ROWS, K, 12, "f64")
        lo, hi = rank * N_ROWS // world, (rank + 1) * N_ROWS // world
        Xp = W[lo:hi].copy()
        Xp[: max(0, M - lo)] = 0.0  # rows of the exact top block are not sketched
        return sk.apply_full(Xp, row0=lo)
    sk = sketch.SRHTSketch(N_ROWS, K, 13)
    Nh = sk.N // world  # world = 2: H_N = H_2 (x) H_{N/2}
    lo = rank * Nh
    xp = np.zeros((Nh, M))
    rows = np.arange(lo, min(lo + Nh, N_ROWS))
    xp[: len(rows)] = W[rows]
    xp[: max(0, M - lo)] = 0.0
    y = sketch.hadamard(xp * math.sqrt(sk.N / sk.k) * sk.signs[lo:lo + Nh, None])
    h2 = np.array([[1.0, 1.0], [1.0, -1.0]]) / math.sqrt(2.0)
    i_hi, i_lo = sk.rows // Nh, sk.rows % Nh
    return h2[i_hi, rank][:, None] * y[i_lo]


def _rank_main(rank, world, port, kind, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        part = torch.tensor(_shard_sketch(rank, world, kind))
        dist.all_reduce(part, op=dist.ReduceOp.SUM)
        out[rank] = part.numpy()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["gaussian", "srht"])
def test_sum_of_shard_sketches_is_the_sketch(kind):
    world, port = 2, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(world, port, kind, out), nprocs=world, join=True)
        got = [np.asarray(out[r]) for r in range(world)]
    W = ri.gaussian(N_ROWS, M, 11)
    sk = sketch.GaussianSketch(N_ROWS, K, 12, "f64") if kind == "gaussian" else sketch.SRHTSketch(N_ROWS, K, 13)
    ref = sketch.rh_sketch(W, M, sk)[M:]
    assert np.array_equal(got[0], got[1])  # every rank holds the same sum
    assert np.max(np.abs(got[0] - ref)) <= 1e-12 * np.abs(ref).max()
