"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the factorisation method: it only draws
test matrices.  The recipes follow the workloads of the paper's experiments
(Section 8) as restated for this project:

* ``gaussian``          W with i.i.d. N(0,1) entries.
* ``spectrum``          W = A diag(sigma) B, A (n x m) and B (m x m) with
                        orthonormal columns (QR of Gaussian matrices), sigma
                        log-spaced from 1 down to 1/cond.
* ``parametric``        the matrix C_m of Section 8, entries
                        f(x, mu) = sin(10 (mu + x)) / (cos(100 (mu - x)) + 1.1).
* ``ragged_batch``      the sizes of a batch of tall-skinny problems, n_i
                        log-uniform in [n_lo, n_hi], m_i drawn from a set.

Each function returns float64 numpy arrays; callers round to the stored dtype.
GPU-resident variants for the full-size benchmark live in ``device``; they use
the same recipe with torch's CUDA generator (different values, same law).
"""

from __future__ import annotations

import numpy as np


def gaussian(n: int, m: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal((n, m))


def orthonormal(n: int, m: int, rng: np.random.Generator) -> np.ndarray:
    q, r = np.linalg.qr(rng.standard_normal((n, m)))
    return q * np.sign(np.diag(r))[None, :]


def log_spectrum(m: int, cond: float) -> np.ndarray:
    return np.logspace(0.0, -np.log10(cond), m)


def spectrum(n: int, m: int, cond: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    A = orthonormal(n, m, rng)
    B = orthonormal(m, m, rng)
    return (A * log_spectrum(m, cond)[None, :]) @ B


def parametric(n: int, m: int) -> np.ndarray:
    x = np.arange(n) / (n - 1)
    mu = np.arange(m) / max(m - 1, 1)
    X, MU = np.meshgrid(x, mu, indexing="ij")
    return np.sin(10.0 * (MU + X)) / (np.cos(100.0 * (MU - X)) + 1.1)


def ragged_batch(count: int, n_lo: int, n_hi: int, m_choices, seed: int):
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), count)).astype(np.int64)
    m = rng.choice(np.asarray(m_choices), count)
    return n, m


def to_dtype(W: np.ndarray, dtype: str) -> np.ndarray:
    """Round a float64 matrix to its stored format (f64 or f32), keep Fortran order."""
    if dtype == "f64":
        return np.asfortranarray(W, dtype=np.float64)
    if dtype == "f32":
        return np.asfortranarray(W, dtype=np.float32)
    raise ValueError(dtype)


# ---------------------------------------------------------------------------
# GPU-resident variants (same recipes; torch's CUDA generator) for full sizes
# ---------------------------------------------------------------------------


def _device_orthonormal(G):
    """Orthonormal columns spanning G (n x m, float64 on the device) by two
    Cholesky-QR passes: the m x m Gram matrices are factored on the host."""
    import torch

    A = G
    for _ in range(2):
        C = (A.t() @ A).cpu().numpy()
        Rinv = np.linalg.inv(np.linalg.cholesky(C).T)
        A = A @ torch.tensor(Rinv, dtype=torch.float64, device=A.device)
    return A


def device_spectrum(n: int, m: int, cond: float, seed: int, dtype=None, device="cuda"):
    """W = A diag(sigma) B built in float64 on the device, returned column-major
    in `dtype` (torch dtype, default float32).  A: orthonormal basis of an n x m
    Gaussian matrix; B: Q factor of an m x m Gaussian matrix (host QR)."""
    import torch

    dtype = dtype or torch.float32
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    A = _device_orthonormal(torch.randn((n, m), generator=g, dtype=torch.float64, device=device))
    Bm = torch.tensor(orthonormal(m, m, np.random.default_rng(seed)), dtype=torch.float64, device=device)
    sig = torch.tensor(log_spectrum(m, cond), dtype=torch.float64, device=device)
    W = (A * sig[None, :]) @ Bm
    del A
    out = torch.empty((m, n), dtype=dtype, device=device).t()
    out.copy_(W)
    return out


def device_gaussian(n: int, m: int, seed: int, dtype=None, device="cuda"):
    import torch

    dtype = dtype or torch.float32
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    out = torch.empty((m, n), dtype=dtype, device=device).t()
    out.copy_(torch.randn((n, m), generator=g, dtype=torch.float64, device=device))
    return out


def device_ragged_batch(count: int, n_lo: int, n_hi: int, m_choices, cond: float, seed: int, dtype=None,
                        device="cuda"):
    """The ragged batch workload on the device: n_i log-uniform in [n_lo, n_hi],
    m_i uniform over m_choices; even i Gaussian, odd i log-spaced spectrum
    1 .. 1/cond.  Returns (list of column-major W_i, n, m)."""
    n, m = ragged_batch(count, n_lo, n_hi, m_choices, seed)
    Ws = []
    for i in range(count):
        ni, mi = int(n[i]), int(m[i])
        if i % 2 == 0:
            Ws.append(device_gaussian(ni, mi, seed * 100003 + i, dtype, device))
        else:
            Ws.append(device_spectrum(ni, mi, cond, seed * 100003 + i, dtype, device))
    return Ws, [int(x) for x in n], [int(x) for x in m]


# ---------------------------------------------------------------------------
# 2-D convection-diffusion operator (the GMRES workload), matrix-free
# ---------------------------------------------------------------------------


def stencil_apply(u, g: int, peclet: float = 10.0):
    """A u for -Laplace(u) + Pe (u_x + u_y) on the unit square, g x g interior
    points, h = 1/(g+1), zero Dirichlet boundary, central differences, scaled by
    h^2.  `u` is a numpy array or torch tensor of length g*g (row-major grid)."""
    c = peclet / (2.0 * (g + 1))  # Pe h / 2
    U = u.reshape(g, g)
    out = 4.0 * U
    out[1:, :] += -U[:-1, :] - c * U[:-1, :]
    out[:-1, :] += -U[1:, :] + c * U[1:, :]
    out[:, 1:] += -U[:, :-1] - c * U[:, :-1]
    out[:, :-1] += -U[:, 1:] + c * U[:, 1:]
    return out.reshape(-1)
