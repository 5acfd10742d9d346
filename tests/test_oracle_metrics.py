"""Pins of the oracle's accuracy measures (oracle/metrics.py) against closed forms.

Each case is built so that its value follows from the definitions alone (the
sketch orthogonality of Thm. mainthm, the relative factorisation error of
Thm. factoerror, the 2-norm condition number, R up to the row signs of the
Householder convention), and so that a plausible slip -- a dropped Omega term,
a Frobenius norm in place of the 2-norm, a transposed factor, signs aligned on
columns instead of rows -- changes the value.
"""

import numpy as np
import pytest

from oracle import metrics, sketch


def _top_block(n, d):
    """Q = [diag(d); 0] (n x len(d)): only the exact top block of Psi sees it."""
    Q = np.zeros((n, len(d)))
    Q[np.arange(len(d)), np.arange(len(d))] = d
    return Q


@pytest.mark.parametrize("kind", ["gaussian", "srht"])
def test_orthogonality_of_scaled_identity_block(kind):
    # Psi [diag(d); 0] = [diag(d); 0] for any Omega (Psi = diag(I_m, Omega)), so
    # (Psi Q)^t Psi Q = diag(d^2) and ||I - diag(d^2)||_2 = max |1 - d_i^2|.
    n, k = 64, 16
    sk = sketch.GaussianSketch(n, k, 5) if kind == "gaussian" else sketch.SRHTSketch(n, k, 5)
    delta = 1e-3
    Q = _top_block(n, [1.0, 1.0, 1.0 + delta])
    assert metrics.sketch_orthogonality(Q, sk) == pytest.approx(2 * delta + delta**2, rel=1e-10)
    # two perturbed columns: the 2-norm takes the larger one; the Frobenius norm
    # would give sqrt(a^2 + b^2)
    Q = _top_block(n, [1.0 + 2e-3, 1.0 - 1e-3, 1.0])
    a, b = 1 - (1 + 2e-3) ** 2, 1 - (1 - 1e-3) ** 2
    assert metrics.sketch_orthogonality(Q, sk) == pytest.approx(max(abs(a), abs(b)), rel=1e-10)
    assert abs(metrics.sketch_orthogonality(Q, sk) - np.hypot(a, b)) > 1e-4
    # exactly orthonormal in the sketch
    assert metrics.sketch_orthogonality(_top_block(n, [1.0, -1.0]), sk) == 0.0


def test_orthogonality_sees_the_omega_rows():
    # Every column of an SRHT Omega_full = sqrt(N/k) P H D has k entries
    # +-sqrt(N/k)/sqrt(N) = +-1/sqrt(k) (Section 2.3), so ||Omega e_j|| = 1.
    # For x = e_0 + t e_j with j >= m: Psi x = [e_0; t Omega e_j] and
    # ||I - (Psi x)^t Psi x|| = |1 - (1 + t^2)| = t^2.  Without the Omega rows it
    # would be 0; with a wrong 1/sqrt scale it would differ from t^2.
    n, k, m = 128, 32, 1
    sk = sketch.SRHTSketch(n, k, 11)
    for j, t in [(5, 0.25), (77, 0.5), (127, 1e-2)]:
        x = np.zeros((n, 1))
        x[0, 0] = 1.0
        x[j, 0] = t
        assert metrics.sketch_orthogonality(x, sk, m=m) == pytest.approx(t * t, rel=1e-12)


def test_orthogonality_two_columns_sharing_omega_rows():
    # Q = [e_0 + t e_j, e_1 + t e_j] (j >= m = 2): (Psi Q)^t Psi Q = I + t^2 1 1^t,
    # whose eigenvalues are 1 and 1 + 2 t^2: the orthogonality is 2 t^2 (an
    # off-diagonal slip would give t^2).
    n, k, m, j, t = 64, 16, 2, 40, 0.3
    sk = sketch.SRHTSketch(n, k, 3)
    Q = np.zeros((n, 2))
    Q[0, 0] = Q[1, 1] = 1.0
    Q[j, :] = t
    assert metrics.sketch_orthogonality(Q, sk, m=m) == pytest.approx(2 * t * t, rel=1e-12)


def test_residual_pythagorean_case():
    # Q = [I_2; 0], R = diag(3, 4) (||QR||_F = 5), and E of Frobenius norm 12 in
    # the rows below 2: W = QR + E has ||W||_F = 13 and ||W - QR||_F / ||W||_F = 12/13.
    n = 10
    Q = _top_block(n, [1.0, 1.0])
    R = np.diag([3.0, 4.0])
    a = np.zeros(n)
    a[5], a[7] = 3.0, 4.0  # ||a|| = 5
    b = np.array([0.6, 0.8]) * (12.0 / 5.0)  # ||b|| = 12/5, so ||a b^t||_F = 12
    W = Q @ R + np.outer(a, b)
    assert metrics.residual(W, Q, R) == pytest.approx(12.0 / 13.0, rel=1e-14)


def test_residual_order_of_the_factors():
    # W = Q R exactly, with R upper triangular and not symmetric: the residual is
    # at rounding level, while Q R^t (a transposed operand) leaves R - R^t.
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((50, 4)))
    R = np.triu(rng.standard_normal((4, 4))) + 4 * np.eye(4)
    W = Q @ R
    assert metrics.residual(W, Q, R) < 1e-15
    want = np.linalg.norm(R.T - R) / np.linalg.norm(R)  # ||Q (R^t - R)||_F = ||R^t - R||_F
    assert metrics.residual(W, Q, R.T) == pytest.approx(want, rel=1e-12)


def test_cond_closed_forms():
    # 2-norm condition number sigma_max / sigma_min
    A = np.zeros((9, 3))
    A[0, 0], A[4, 1], A[8, 2] = 10.0, -1.0, 1e-3
    assert metrics.cond(A) == pytest.approx(1e4, rel=1e-12)
    # orthonormal columns: 1
    Q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((20, 5)))
    assert metrics.cond(Q) == pytest.approx(1.0, abs=1e-14)
    # diag(1, 1, 1, 1/2): 2 (a Frobenius-based estimate ||A||_F ||A^+||_F would be
    # sqrt(3.25) sqrt(7) ~ 4.77)
    assert metrics.cond(np.diag([1.0, 1.0, 1.0, 0.5])) == pytest.approx(2.0, rel=1e-14)
    # [[1, 1], [0, 1]]: sigma = (sqrt 5 +- 1) / 2, cond = (3 + sqrt 5) / 2
    assert metrics.cond(np.array([[1.0, 1.0], [0.0, 1.0]])) == pytest.approx((3 + 5**0.5) / 2, rel=1e-14)


def test_r_relative_difference_row_signs():
    Rref = np.array([[2.0, -1.0, 3.0], [0.0, -4.0, 0.5], [0.0, 0.0, 1.5]])
    D = np.diag([-1.0, 1.0, -1.0])
    # R differing from Rref only by the signs of its rows: 0
    assert metrics.r_relative_difference(D @ Rref, Rref) == 0.0
    # aligning column signs instead would leave D Rref D - Rref != 0
    assert np.linalg.norm(D @ Rref @ D - Rref) > 1
    # a perturbation eps of one entry of a flipped row: eps / ||Rref||_F
    eps = 1e-6
    R = D @ Rref
    R[0, 2] += eps
    assert metrics.r_relative_difference(R, Rref) == pytest.approx(eps / np.linalg.norm(Rref), rel=1e-8)
    # a genuinely different R: the sign alignment uses the diagonals only
    R2 = Rref.copy()
    R2[1, 2] = -R2[1, 2]
    assert metrics.r_relative_difference(R2, Rref) == pytest.approx(
        2 * abs(Rref[1, 2]) / np.linalg.norm(Rref), rel=1e-14
    )
