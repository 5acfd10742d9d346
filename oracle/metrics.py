"""Accuracy measures, computed in FP64 on the host (oracle side).

* sketch orthogonality  ||I - (Psi Q)^t (Psi Q)||_2  (Thm. mainthm: Psi Q has
  orthonormal columns), with Psi Q recomputed here in FP64 from the same Psi;
* relative factorisation error ||W - Q R||_F / ||W||_F (Thm. factoerror);
* condition number of Q (Thm. conditionnumberQ);
* R agreement up to the row signs of the Householder convention.
"""

from __future__ import annotations

import numpy as np

from .sketch import rh_sketch


def sketch_orthogonality(Q, sk, m: int | None = None) -> float:
    Q = np.asarray(Q, dtype=np.float64)
    m = Q.shape[1] if m is None else m
    PQ = rh_sketch(Q, m, sk)
    G = PQ.T @ PQ
    E = np.eye(G.shape[0]) - G
    return float(np.max(np.abs(np.linalg.eigvalsh((E + E.T) / 2))))


def residual(W, Q, R) -> float:
    W = np.asarray(W, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    return float(np.linalg.norm(W - Q @ R) / np.linalg.norm(W))


def cond(A) -> float:
    s = np.linalg.svd(np.asarray(A, dtype=np.float64), compute_uv=False)
    return float(s[0] / s[-1])


def r_relative_difference(R, Rref) -> float:
    """||D R - Rref||_F / ||Rref||_F with D = diag(sign) aligning the diagonals."""
    R = np.asarray(R, dtype=np.float64)
    Rref = np.asarray(Rref, dtype=np.float64)
    d = np.sign(np.diag(R)) * np.sign(np.diag(Rref))
    d[d == 0] = 1
    return float(np.linalg.norm(d[:, None] * R - Rref) / np.linalg.norm(Rref))
