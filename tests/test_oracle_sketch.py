"""Pins of the oracle's sketches: Walsh-Hadamard, SRHT, Gaussian, RHSketch."""

import math
import os

import numpy as np
import pytest

from oracle import rng, sketch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def sylvester(N):
    return np.array([[(-1) ** bin(i & j).count("1") for j in range(N)] for i in range(N)], dtype=np.float64)


def test_hadamard_golden_8():
    rows = [ln for ln in open(os.path.join(GOLDEN, "hadamard8_sylvester.txt")) if not ln.startswith("#")]
    H8 = np.array([[float(v) for v in r.split()] for r in rows if r.strip()])
    assert np.array_equal(sketch.hadamard_unnormalised(np.eye(8)), H8)


@pytest.mark.parametrize("N", [1, 2, 4, 8, 16, 32, 64])
def test_hadamard_equals_brute_force(N):
    got = sketch.hadamard(np.eye(N))
    assert np.max(np.abs(got - sylvester(N) / math.sqrt(N))) < 1e-15
    assert np.array_equal(sketch.hadamard_unnormalised(np.eye(N)), sylvester(N))


def test_hadamard_is_an_involution_and_isometry():
    x = np.random.default_rng(0).standard_normal((1024, 3))
    y = sketch.hadamard(x)
    assert np.allclose(np.linalg.norm(y, axis=0), np.linalg.norm(x, axis=0), rtol=1e-14)
    assert np.max(np.abs(sketch.hadamard(y) - x)) < 1e-13


def test_hadamard_kronecker_split():
    # H_N = H_{N1} (x) H_{N2} in Sylvester order: x viewed as (N1, N2) row-major
    N1, N2 = 8, 32
    x = np.random.default_rng(1).standard_normal(N1 * N2)
    direct = sketch.hadamard_unnormalised(x)
    two_stage = (sylvester(N1) @ x.reshape(N1, N2) @ sylvester(N2).T).ravel()
    assert np.max(np.abs(direct - two_stage)) < 1e-12


@pytest.mark.parametrize("n,k", [(64, 8), (50, 16), (33, 33)])
def test_srht_explicit_matrix(n, k):
    sk = sketch.SRHTSketch(n, k, seed=5)
    N = sketch.next_pow2(n)
    P = np.eye(N)[sk.rows]
    D = np.diag(sk.signs)
    H = sylvester(N) / math.sqrt(N)
    want = math.sqrt(N / k) * P @ H @ D
    assert np.max(np.abs(sk.full_matrix() - want[:, :n])) < 1e-14


def test_srht_full_sample_is_orthogonal_up_to_scale():
    n = k = 64
    sk = sketch.SRHTSketch(n, k, seed=9)
    x = np.random.default_rng(2).standard_normal(n)
    assert abs(np.linalg.norm(sk.apply_full(x)) - np.linalg.norm(x)) < 1e-13


def test_gaussian_sketch_entries():
    n, k = 300, 40
    sk = sketch.GaussianSketch(n, k, seed=3, dtype="f64")
    Om = sk.full_matrix()
    G = np.array([[rng.gaussian_values(3, np.array([r * n + c], dtype=np.uint64))[0] for c in range(n)] for r in range(k)])
    assert np.array_equal(Om, G / math.sqrt(k))
    x = np.random.default_rng(4).standard_normal(n)
    assert np.max(np.abs(sk.apply_full(x) - Om @ x)) < 1e-13
    bf = sketch.GaussianSketch(n, k, seed=3, dtype="bf16")
    assert np.array_equal(bf.G_block(0, n), rng.round_to_dtype(G, "bf16"))
    assert np.array_equal(bf.full_matrix(), rng.round_to_dtype(G, "bf16") / math.sqrt(k))


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
def test_rh_sketch_structure(kind):
    n, m, k = 100, 7, 24
    sk = sketch.SRHTSketch(n, k, 1) if kind == "srht" else sketch.GaussianSketch(n, k, 1)
    X = np.random.default_rng(5).standard_normal((n, 3))
    Z = sketch.rh_sketch(X, m, sk)
    assert Z.shape == (k + m, 3)
    assert np.array_equal(Z[:m], X[:m])  # exact copy of the top block
    Psi = sketch.psi_matrix(sk, m)
    assert np.max(np.abs(Z - Psi @ X)) < 1e-13
    e = np.zeros(n)
    e[2] = 1
    assert np.linalg.norm(sketch.rh_sketch(e, m, sk)) == 1.0  # ||Psi e_j|| = 1, j < m


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
def test_epsilon_embedding_of_an_orthonormal_basis(kind):
    # Section 8: cond(Psi Q) = 1 + O(eps) for an exact orthonormal basis
    n, m, k = 4096, 32, 256
    Q = np.linalg.qr(np.random.default_rng(6).standard_normal((n, m)))[0]
    sk = sketch.SRHTSketch(n, k, 2) if kind == "srht" else sketch.GaussianSketch(n, k, 2)
    s = np.linalg.svd(sketch.rh_sketch(Q, m, sk), compute_uv=False)
    # an epsilon-embedding with epsilon = 1/2 (k = 8 m), hence Cond <= 3 (Section 2.3)
    assert 0.5 < s[-1] and s[0] < 1.5 and s[0] / s[-1] < 3.0
