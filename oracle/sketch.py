"""Sketching operators and RHSketch (oracle side).

* Walsh-Hadamard transform in Sylvester (natural) order: the recursion
  H_{p+1} = [[H_p, H_p], [H_p, -H_p]] of the SRHT lemma's proof (appendix),
  normalised by 1/sqrt(N) in one step at the end.
* SRHT  Omega = sqrt(N/k) P H D  (Section 2.3), applied in the order of
  Lemma "srht" (Section 4): scale, flip signs, Hadamard transform, sample.
  For n not a power of two the input is zero-padded to N = 2^ceil(log2 n).
* Gaussian Omega = G / sqrt(k) with G i.i.d. N(0,1) (Section 2.3).
* Psi = diag(I_m, Omega) of eq. (psi) and RHSketch (Algorithm 1).

Reading of the dimensions.  Section 2.1 puts Omega in R^{l x (n-m)} and Psi in
R^{(l+m) x n}.  A sketch is created for a row count n and a sketch size k
without knowing m; the operator Omega_full (k x n, or k x N for the SRHT) is
drawn once and, for a factorisation with m columns, Omega := the columns
m..n-1 of Omega_full.  For the SRHT this is the same as zeroing the first m
entries of the length-N input before the transform.  l = k.
"""

from __future__ import annotations

import math

import numpy as np

from . import rng


def next_pow2(n: int) -> int:
    return 1 << max(0, (int(n) - 1).bit_length())


def _one_of(arr):
    """1 in the arithmetic of array ``arr`` (a decimal if it holds decimals)."""
    if arr.dtype != object:
        return 1.0
    for v in arr.flat:
        if not isinstance(v, int):
            return v * 0 + 1
    return 1


def _sqrt(x):
    """sqrt for float or decimal scalars (object arrays use the element's method)."""
    if hasattr(x, "sqrt"):
        return x.sqrt()
    return math.sqrt(x)


def hadamard_unnormalised(x: np.ndarray) -> np.ndarray:
    """H_p x for x of shape (N, c), N = 2^p, by the Sylvester recursion: the two
    halves are transformed first, then combined as (a + b; a - b)."""
    x = np.asarray(x)
    N = x.shape[0]
    if N & (N - 1):
        raise ValueError("length must be a power of two")
    y = x.reshape(N, -1).copy()
    c = y.shape[1]
    h = 1
    while h < N:
        y = y.reshape(N // (2 * h), 2, h, c)
        a = y[:, 0]
        b = y[:, 1]
        y = np.stack([a + b, a - b], axis=1).reshape(N, c)
        h *= 2
    return y.reshape(x.shape)


def hadamard(x: np.ndarray) -> np.ndarray:
    """Normalised Walsh-Hadamard transform H x = 2^{-p/2} H_p x."""
    N = x.shape[0]
    one = _one_of(x)
    scale = one / _sqrt(one * N)
    return hadamard_unnormalised(x) * scale


class SRHTSketch:
    """Omega_full = sqrt(N/k) P H D, a k x N operator on zero-padded inputs."""

    kind = "srht"

    def __init__(self, n: int, k: int, seed: int):
        self.n, self.k, self.seed = int(n), int(k), int(seed)
        self.N = next_pow2(self.n)
        if not 0 < self.k <= self.N:
            raise ValueError("need 0 < k <= N")
        self.signs = rng.srht_signs(self.seed, self.N)
        self.rows = rng.srht_sample(self.seed, self.N, self.k)

    def apply_full(self, X: np.ndarray) -> np.ndarray:
        """Omega_full X for X with n rows (or N rows), shape (k, c)."""
        X = np.asarray(X)
        squeeze = X.ndim == 1
        X = X.reshape(X.shape[0], -1)
        pad = np.zeros((self.N, X.shape[1]), dtype=X.dtype)
        pad[: X.shape[0]] = X
        one = _one_of(X)
        pad[X.shape[0]:] = one * 0
        y = pad * _sqrt(one * self.N / self.k)  # scale
        sg = self.signs.astype(np.int64).astype(object) if pad.dtype == object else self.signs
        y = y * sg[:, None]  # flip signs (exact)
        y = hadamard(y)  # normalised Hadamard transform
        y = y[self.rows]  # sample (exact)
        return y[:, 0] if squeeze else y

    def full_matrix(self) -> np.ndarray:
        return self.apply_full(np.eye(self.n))


class GaussianSketch:
    """Omega_full = G / sqrt(k), G a k x n matrix of seeded N(0,1) values rounded
    to the storage format ``dtype`` (f64, f32, bf16 or f16)."""

    kind = "gaussian"
    CHUNK = 1 << 14

    def __init__(self, n: int, k: int, seed: int, dtype: str = "f64"):
        self.n, self.k, self.seed, self.dtype = int(n), int(k), int(seed), dtype

    def G_block(self, c0: int, c1: int) -> np.ndarray:
        return rng.gaussian_block(self.seed, self.n, np.arange(self.k), np.arange(c0, c1), self.dtype)

    def omega_block(self, c0: int, c1: int) -> np.ndarray:
        return self.G_block(c0, c1) / math.sqrt(self.k)

    def apply_full(self, X: np.ndarray, row0: int = 0) -> np.ndarray:
        """Omega_full[:, row0:row0+len(X)] X, generated in column chunks."""
        X = np.asarray(X, dtype=np.float64)
        squeeze = X.ndim == 1
        X = X.reshape(X.shape[0], -1)
        out = np.zeros((self.k, X.shape[1]))
        for c0 in range(0, X.shape[0], self.CHUNK):
            c1 = min(X.shape[0], c0 + self.CHUNK)
            out += self.omega_block(row0 + c0, row0 + c1) @ X[c0:c1]
        return out[:, 0] if squeeze else out

    def full_matrix(self) -> np.ndarray:
        return self.omega_block(0, self.n)


class ExplicitSketch:
    """A given Omega_full matrix (tests: integer or decimal entries, Psi = I, ...)."""

    kind = "explicit"

    def __init__(self, omega_full: np.ndarray):
        self.omega = np.asarray(omega_full)
        self.k, self.n = self.omega.shape

    def apply_full(self, X: np.ndarray) -> np.ndarray:
        return self.omega @ X

    def full_matrix(self) -> np.ndarray:
        return self.omega


def identity_sketch(n: int, m: int, dtype=np.float64) -> ExplicitSketch:
    """Omega_full whose columns m..n-1 form I_{n-m}: Psi_m = I_n (so RHQR is HQR)."""
    om = np.zeros((n - m, n), dtype=dtype)
    for i in range(n - m):
        om[i, m + i] = 1
    if dtype == object:
        om = om.astype(object)
    return ExplicitSketch(om)


def apply_tail(sk, X_tail: np.ndarray, m: int) -> np.ndarray:
    """Omega X_tail with Omega = columns m..n-1 of Omega_full (X_tail has n-m rows)."""
    if isinstance(sk, GaussianSketch):
        return sk.apply_full(X_tail, row0=m)
    if isinstance(sk, ExplicitSketch):
        return sk.omega[:, m:] @ X_tail
    full = np.zeros((m + X_tail.shape[0],) + X_tail.shape[1:], dtype=X_tail.dtype)
    full[:m] = _one_of(X_tail) * 0
    full[m:] = X_tail
    return sk.apply_full(full)


def rh_sketch(X: np.ndarray, m: int, sk) -> np.ndarray:
    """Algorithm 1 (RHSketch): Psi X = [X_{1:m}; Omega X_{m+1:n}], shape (k+m, c).
    Omega = Omega_full restricted to the columns m..n-1."""
    X = np.asarray(X)
    squeeze = X.ndim == 1
    X2 = X.reshape(X.shape[0], -1)
    out = np.concatenate([X2[:m], apply_tail(sk, X2[m:], m)], axis=0)
    return out[:, 0] if squeeze else out


def psi_matrix(sk, m: int) -> np.ndarray:
    """Explicit Psi_m = diag(I_m, Omega) of eq. (psi), (k+m) x n (small n only)."""
    om = np.asarray(sk.full_matrix())
    n = sk.n
    om = om[:, :n].copy()
    om[:, :m] = 0
    top = np.zeros((m, n), dtype=om.dtype)
    for i in range(m):
        top[i, i] = 1
    return np.concatenate([top, om], axis=0)
