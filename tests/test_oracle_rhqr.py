"""Pins of the oracle's factorisations against what the paper and mathematics fix."""

import decimal
import math

import numpy as np
import pytest

import rhqr_inputs as ri
from oracle import metrics, rhqr, sketch

D = decimal.Decimal


def dec(a):
    return np.vectorize(lambda v: D(int(v)) if float(v).is_integer() else D(repr(float(v))), otypes=[object])(a)


def explicit_reflector(u, Psi):
    """P(u, Psi) = I - 2/||Psi u||^2 u (Psi u)^t Psi  (eq. basereflector)."""
    s = Psi @ u
    return np.eye(len(u)) - (2.0 / (s @ s)) * np.outer(u, s @ Psi)


# ---------------------------------------------------------------------------
# Algorithm 2
# ---------------------------------------------------------------------------


def test_rh_vector_closed_form_identity_sketch():
    # Psi = I (n = 2, m = 1): a = 3, rho = 5, sigma = +1, gamma = 8
    w = np.array([3.0, 4.0])
    u, s, sigma, rho, beta = rhqr.rh_vector(w, w.copy(), 0)
    assert (sigma, rho, beta) == (1, 5.0, 1.6)
    assert np.array_equal(u, [1.0, 0.5]) and np.array_equal(s, u)
    # the norm scaling: ||s||^2 = 2, beta = 1
    u2, s2, _, _, b2 = rhqr.rh_vector(w, w.copy(), 0, "norm")
    assert b2 == 1.0 and abs(s2 @ s2 - 2.0) < 1e-15


def test_rh_vector_closed_form_with_sketch():
    # n = 3, m = 1, Omega = [1 1]: Psi w = (w1, w2 + w3); w = (-1, 2, 2) -> y = (-1, 4)
    sk = sketch.ExplicitSketch(np.array([[0.0, 1.0, 1.0]]))
    w = np.array([-1.0, 2.0, 2.0])
    y = sketch.rh_sketch(w, 1, sk)
    u, s, sigma, rho, beta = rhqr.rh_vector(w, y, 0)
    r17 = math.sqrt(17.0)
    assert sigma == -1 and abs(rho - r17) < 1e-15
    gamma = -1 - r17
    assert np.allclose(u, [1.0, 2 / gamma, 2 / gamma], rtol=1e-15)
    assert abs(beta - (1 + 1 / r17)) < 1e-15
    Psi = sketch.psi_matrix(sk, 1)
    Pw = explicit_reflector(u, Psi) @ w
    assert np.allclose(Pw, [-sigma * rho, 0.0, 0.0], atol=1e-14)  # eq. (sumup)


@pytest.mark.parametrize("scaling", ["unit", "norm"])
@pytest.mark.parametrize("j", [0, 2, 4])
def test_rh_vector_elimination_property(scaling, j):
    n, m, k = 40, 5, 12
    sk = sketch.GaussianSketch(n, k, 7)
    Psi = sketch.psi_matrix(sk, m)
    w = np.random.default_rng(j).standard_normal(n)
    u, s, sigma, rho, beta = rhqr.rh_vector(w, Psi @ w, j, scaling)
    assert np.max(np.abs(s - Psi @ u)) < 1e-14  # s = Psi u
    assert abs(beta - 2 / (s @ s)) < 1e-14
    Pw = explicit_reflector(u, Psi) @ w
    want = np.concatenate([w[:j], [-sigma * rho], np.zeros(n - j - 1)])
    assert np.max(np.abs(Pw - want)) < 1e-13
    if scaling == "unit":
        assert u[j] == 1.0 and np.all(u[:j] == 0)


def test_rh_vector_sign_of_zero_and_breakdown():
    w = np.array([0.0, 3.0, 4.0])
    u, s, sigma, rho, beta = rhqr.rh_vector(w, w.copy(), 0)
    assert sigma == 1 and rho == 5.0 and beta == 1.0
    with pytest.raises(rhqr.Breakdown):
        rhqr.rh_vector(np.zeros(3), np.zeros(3), 1)


# ---------------------------------------------------------------------------
# Theorem "mainthm" and the compact forms
# ---------------------------------------------------------------------------


def _case(kind, n=256, m=8, k=32, seed=0):
    W = ri.gaussian(n, m, seed)
    sk = sketch.SRHTSketch(n, k, seed + 1) if kind == "srht" else sketch.GaussianSketch(n, k, seed + 1)
    return W, sk


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
def test_main_theorem_against_lapack(kind):
    W, sk = _case(kind)
    m = W.shape[1]
    U, S, T, R = rhqr.rhqr_left(W, sk)
    Q = rhqr.form_q(U, T)
    Z = sketch.rh_sketch(W, m, sk)
    QL, RL = np.linalg.qr(Z)  # LAPACK Householder QR of Psi W
    d = np.sign(np.diag(R)) * np.sign(np.diag(RL))
    assert np.max(np.abs(d[:, None] * R - RL)) < 1e-13 * np.abs(RL).max()
    assert np.max(np.abs(sketch.rh_sketch(Q, m, sk) * d[None, :] - QL)) < 1e-13
    assert metrics.sketch_orthogonality(Q, sk) < 1e-14
    assert metrics.residual(W, Q, R) < 1e-14
    assert np.allclose(R, np.triu(R))
    assert np.max(np.abs(S - sketch.rh_sketch(U, m, sk))) < 1e-13  # S = Psi U
    U1 = U[:m]
    assert np.allclose(U1, np.tril(U1)) and np.all(np.diag(U1) == 1.0)


def test_compact_form_equals_product_of_reflectors():
    n, m, k = 48, 4, 10
    W, sk = _case("gaussian", n, m, k, 3)
    U, S, T, R = rhqr.rhqr_left(W, sk)
    Psi = sketch.psi_matrix(sk, m)
    prod = np.eye(n)
    for j in range(m):
        prod = prod @ explicit_reflector(U[:, j], Psi)
    assert np.max(np.abs(prod - (np.eye(n) - U @ T @ S.T @ Psi))) < 1e-13
    prod_rev = np.eye(n)
    for j in reversed(range(m)):
        prod_rev = prod_rev @ explicit_reflector(U[:, j], Psi)
    assert np.max(np.abs(prod_rev - (np.eye(n) - U @ T.T @ S.T @ Psi))) < 1e-13
    # P_m ... P_1 W = [R; 0] (eq. triangularization)
    RW = prod_rev @ W
    assert np.max(np.abs(RW[:m] - R)) < 1e-13 and np.max(np.abs(RW[m:])) < 1e-13
    # Woodbury: (Psi U)^t Psi U = T^{-1} + T^{-t}  (eq. generalwoodburry)
    Ti = np.linalg.inv(T)
    assert np.max(np.abs(S.T @ S - Ti - Ti.T)) < 1e-12


@pytest.mark.parametrize("kind", ["srht", "gaussian"])
def test_right_left_and_reconstructed_agree(kind):
    W, sk = _case(kind, 300, 10, 40, 5)
    m = W.shape[1]
    UL, SL, TL, RL = rhqr.rhqr_left(W, sk)
    UR, SR, TR, RR = rhqr.rhqr_right(W, sk)
    UC, SC, TC, RC, M = rhqr.rec_rhqr(W, sk)
    for A, B in [(UL, UR), (UL, UC), (SL, SR), (SL, SC), (TL, TR), (TL, TC)]:
        assert np.max(np.abs(A - B)) < 1e-12 * max(1, np.abs(A).max())
    for A in (RR, RC):
        assert np.max(np.abs(A - RL)) < 1e-12 * np.abs(RL).max()
    # Section 3.3: T^t (Psi U)^t Psi W = -T U_1^t R (upper triangular)
    assert np.max(np.abs(M + TL @ UL[:m].T @ RL)) < 1e-12 * np.abs(M).max()
    full = TC.T @ SC.T @ sketch.rh_sketch(W, m, sk)
    assert np.max(np.abs(np.tril(full, -1))) < 1e-12 * np.abs(full).max()


def test_identity_sketch_is_householder_qr():
    n, m = 30, 6
    W = ri.gaussian(n, m, 8)
    U, S, T, R = rhqr.rhqr_left(W, sketch.identity_sketch(n, m))
    S2, T2, R2 = rhqr.householder_qr(W)
    assert np.max(np.abs(R - R2)) < 1e-13 and np.max(np.abs(U - S2)) < 1e-13
    RL = np.linalg.qr(W)[1]
    assert metrics.r_relative_difference(R, RL) < 1e-14
    Q = rhqr.form_q(U, T)
    assert np.max(np.abs(Q.T @ Q - np.eye(m))) < 1e-14


def test_householder_qr_matches_lapack():
    Z = ri.spectrum(200, 12, 1e6, 9)
    S, T, R = rhqr.householder_qr(Z)
    assert metrics.r_relative_difference(R, np.linalg.qr(Z)[1]) < 1e-14
    Q = np.eye(200, 12) - S @ T @ S[:12].T
    assert np.max(np.abs(Q.T @ Q - np.eye(12))) < 1e-14


def test_lu_characterisation_recovers_the_reflectors():
    W, sk = _case("srht", 200, 6, 24, 11)
    U, S, T, R = rhqr.rhqr_left(W, sk)
    Q = rhqr.form_q(U, T)
    U2, S2, T2 = rhqr.lu_reconstruct(Q, sk)
    assert np.max(np.abs(U2 - U)) < 1e-12 and np.max(np.abs(T2 - T)) < 1e-12
    assert np.max(np.abs(S2 - S)) < 1e-12


# ---------------------------------------------------------------------------
# exact arithmetic on tiny integer inputs (60 significant digits)
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("algo", ["left", "right", "rec"])
def test_exact_arithmetic_on_integer_inputs(algo):
    decimal.getcontext().prec = 60
    r = np.random.default_rng(12)
    n, m, k = 9, 3, 4
    W = dec(r.integers(-5, 6, (n, m)))
    Om = dec(r.integers(-2, 3, (k, n)))
    sk = sketch.ExplicitSketch(Om)
    if algo == "left":
        U, S, T, R = rhqr.rhqr_left(W, sk)
    elif algo == "right":
        U, S, T, R = rhqr.rhqr_right(W, sk)
    else:
        U, S, T, R, _ = rhqr.rec_rhqr(W, sk)
    Q = rhqr.form_q(U, T)
    E = W - Q @ R
    assert max(abs(v) for v in E.ravel()) < D("1e-50")
    PQ = sketch.rh_sketch(Q, m, sk)
    G = PQ.T @ PQ
    for i in range(m):
        for j in range(m):
            assert abs(G[i, j] - (1 if i == j else 0)) < D("1e-50")
    # R agrees with LAPACK on the float64 copy (R is unique up to row signs)
    Rf = R.astype(float)
    RL = np.linalg.qr(sketch.rh_sketch(W.astype(float), m, sketch.ExplicitSketch(Om.astype(float))))[1]
    assert metrics.r_relative_difference(Rf, RL) < 1e-14


def test_exact_arithmetic_srht():
    decimal.getcontext().prec = 60
    n, m, k = 16, 3, 4  # sqrt(N/k)/sqrt(N) = 1/2: exact
    sk = sketch.SRHTSketch(n, k, 3)
    W = dec(np.random.default_rng(13).integers(-4, 5, (n, m)))
    U, S, T, R = rhqr.rhqr_left(W, sk)
    Q = rhqr.form_q(U, T)
    assert max(abs(v) for v in (W - Q @ R).ravel()) < D("1e-50")
    PQ = sketch.rh_sketch(Q, m, sk)
    assert max(abs(v) for v in (PQ.T @ PQ - np.eye(m, dtype=np.int64).astype(object)).ravel()) < D("1e-50")


# ---------------------------------------------------------------------------
# refinement, condition-number independence
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("cond", [1e2, 1e8, 1e12])
def test_left_looking_is_cond_independent(cond):
    W = ri.spectrum(2000, 16, cond, 14)
    sk = sketch.SRHTSketch(2000, 64, 15)
    U, S, T, R = rhqr.rhqr_left(W, sk)
    Q = rhqr.form_q(U, T)
    assert metrics.sketch_orthogonality(Q, sk) < 1e-13
    assert metrics.residual(W, Q, R) < 1e-14
    assert metrics.cond(Q) < 3


def test_refinement_reaches_orthogonality_at_high_condition():
    W = ri.spectrum(2000, 16, 1e12, 16)
    sk = sketch.GaussianSketch(2000, 64, 17)
    Q1, R1, *_ = rhqr.rec_rhqr_refined(W, sk, passes=1)
    Q2, R2, U, S, T = rhqr.rec_rhqr_refined(W, sk, passes=2)
    assert metrics.sketch_orthogonality(Q2, sk) < 1e-13
    assert metrics.sketch_orthogonality(Q2, sk) <= metrics.sketch_orthogonality(Q1, sk)
    assert metrics.residual(W, Q2, R2) < 1e-14
    assert np.max(np.abs(rhqr.form_q(U, T) - Q2)) < 1e-14
    # the last pass's reflectors triangularise W: P_m ... P_1 W = [R; 0]
    RW = rhqr.compact_apply(U, T, S, sk, W, 16, transpose=True)
    assert np.max(np.abs(RW[:16] - R2)) < 1e-12 and np.max(np.abs(RW[16:])) < 1e-12


# ---------------------------------------------------------------------------
# Algorithms 7 and 8
# ---------------------------------------------------------------------------


def _operator(n, seed):
    A = np.random.default_rng(seed).standard_normal((n, n)) / math.sqrt(n) + 2 * np.eye(n)
    return A, (lambda x: A @ x)


def test_arnoldi_relation_and_sketch_orthogonality():
    n, mm, k = 300, 12, 60
    A, Aop = _operator(n, 20)
    sk = sketch.SRHTSketch(n, k, 21)
    b = np.random.default_rng(22).standard_normal(n)
    H, Q, h0, arn = rhqr.rhqr_arnoldi(Aop, b, np.zeros(n), sk, mm)
    assert np.max(np.abs(A @ Q[:, :mm] - Q @ H)) < 1e-12  # eq. (arnoldirelation)
    assert np.allclose(H, np.triu(H, -1))
    PQ = sketch.rh_sketch(Q, mm + 1, sk)
    assert np.max(np.abs(PQ.T @ PQ - np.eye(mm + 1))) < 1e-13
    assert np.max(np.abs(h0[0] * Q[:, 0] - b)) < 1e-13  # r_0 = h_0 q_1


def test_arnoldi_with_identity_sketch_is_textbook_arnoldi():
    n, mm = 60, 8
    A, Aop = _operator(n, 23)
    b = np.random.default_rng(24).standard_normal(n)
    H, Q, h0, _ = rhqr.rhqr_arnoldi(Aop, b, np.zeros(n), sketch.identity_sketch(n, mm + 1), mm)
    # modified Gram-Schmidt Arnoldi (orthonormal basis, unique up to signs)
    V = np.zeros((n, mm + 1))
    Hm = np.zeros((mm + 1, mm))
    V[:, 0] = b / np.linalg.norm(b)
    for j in range(mm):
        w = A @ V[:, j]
        for i in range(j + 1):
            Hm[i, j] = w @ V[:, i]
            w = w - Hm[i, j] * V[:, i]
        Hm[j + 1, j] = np.linalg.norm(w)
        V[:, j + 1] = w / Hm[j + 1, j]
    d = np.sign(np.sum(Q * V, axis=0))
    assert np.max(np.abs(Q * d - V)) < 1e-12
    assert np.max(np.abs(d[:, None] * H * d[None, :mm] - Hm)) < 1e-12


def test_gmres_sketched_optimality_brute_force():
    n, mm, k = 200, 10, 50
    A, Aop = _operator(n, 25)
    sk = sketch.GaussianSketch(n, k, 26)
    b = np.random.default_rng(27).standard_normal(n)
    x0 = np.random.default_rng(28).standard_normal(n) * 0.1
    x, H, Q, h0 = rhqr.rhqr_gmres(Aop, b, x0, sk, mm)
    # brute force: argmin over x0 + K_m(A, r0) of ||Psi (b - A x)||  (eq. rgmresopti)
    r0 = b - A @ x0
    K = np.zeros((n, mm))
    v = r0.copy()
    for j in range(mm):
        K[:, j] = v / np.linalg.norm(v)
        v = A @ K[:, j]
    Kb = np.linalg.qr(K)[0]
    Psi = sketch.psi_matrix(sk, mm + 1)
    c = np.linalg.lstsq(Psi @ A @ Kb, Psi @ r0, rcond=None)[0]
    assert np.max(np.abs(x - (x0 + Kb @ c))) < 1e-10 * np.abs(x).max()


def test_panel_t_inverse_is_diag_inv_beta_plus_striu_gram():
    """The blocked Householder QR never forms a panel's T: T^{-1} =
    diag(1/beta) + striu(V^t V) (eq. generalwoodburry with Psi = I), and
    T^t w is found by forward substitution with its transpose."""
    rng = np.random.default_rng(21)
    Z = rng.standard_normal((60, 12)) @ np.diag(np.logspace(0, -6, 12))
    for scaling in ("unit", "norm"):
        V, T, R = rhqr.householder_qr(Z, scaling)
        beta = np.diag(T)
        M = np.diag(1.0 / beta) + np.triu(V.T @ V, 1)
        assert np.max(np.abs(np.linalg.inv(T) - M)) <= 1e-12 * np.abs(M).max()
        w = rng.standard_normal(12)
        w2 = np.zeros(12)
        for q in range(12):  # forward substitution, M^t upper -> lower
            w2[q] = beta[q] * (w[q] - M[:q, q] @ w2[:q])
        assert np.max(np.abs(w2 - T.T @ w)) <= 1e-12 * np.abs(T.T @ w).max()


# ---------------------------------------------------------------------------
# Algorithm 5 (blockRHQR)
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("kind,bs", [("gaussian", 4), ("srht", 3), ("srht", 12)])
def test_block_rhqr_equals_left_looking(kind, bs):
    W, sk = _case(kind, 300, 12, 40, 31)
    U, S, T, R = rhqr.rhqr_left(W, sk)
    RB, blocks = rhqr.block_rhqr(W, sk, bs)
    scale = np.abs(R).max()
    assert np.max(np.abs(RB - R)) <= 1e-12 * scale
    for c0, Ub, Sb, Tb in blocks:
        b = Ub.shape[1]
        assert np.max(np.abs(Ub - U[:, c0:c0 + b])) <= 1e-11
        assert np.max(np.abs(Sb - S[:, c0:c0 + b])) <= 1e-11
        assert np.max(np.abs(Tb - T[c0:c0 + b, c0:c0 + b])) <= 1e-11
    # W = prod_j (I - U^(j) T^(j) S^(j)t Psi) [R; 0]
    Psi = sketch.psi_matrix(sk, W.shape[1])
    P = np.eye(W.shape[0])
    for _, Ub, Sb, Tb in blocks:
        P = P @ (np.eye(W.shape[0]) - Ub @ Tb @ Sb.T @ Psi)
    RW = np.zeros_like(W)
    RW[: W.shape[1]] = RB
    assert np.max(np.abs(P @ RW - W)) <= 1e-12 * np.abs(W).max()


def test_block_rhqr_exact_arithmetic():
    decimal.getcontext().prec = 60
    r = np.random.default_rng(32)
    n, m, k = 10, 4, 6
    W = dec(r.integers(-5, 6, (n, m)))
    sk = sketch.ExplicitSketch(dec(r.integers(-2, 3, (k, n))))
    U, S, T, R = rhqr.rhqr_left(W, sk)
    RB, blocks = rhqr.block_rhqr(W, sk, 2)
    assert max(abs(v) for v in (RB - R).ravel()) < D("1e-50")
    for c0, Ub, _, Tb in blocks:
        assert max(abs(v) for v in (Ub - U[:, c0:c0 + 2]).ravel()) < D("1e-50")
        assert max(abs(v) for v in (Tb - T[c0:c0 + 2, c0:c0 + 2]).ravel()) < D("1e-50")


# ---------------------------------------------------------------------------
# Algorithm 9 (BLAS2-RGS)
# ---------------------------------------------------------------------------


def test_blas2_rgs_equals_rgs_and_t_is_identity_in_exact_arithmetic():
    decimal.getcontext().prec = 60
    r = np.random.default_rng(41)
    n, m, k = 12, 4, 7
    W = dec(r.integers(-5, 6, (n, m)))
    Om = dec(r.integers(-2, 3, (k, n)))
    Q, R, S, T = rhqr.blas2_rgs(W, Om)
    Qr, Rr = rhqr.rgs(W, Om)
    assert max(abs(v) for v in (Q - Qr).ravel()) < D("1e-50")
    assert max(abs(v) for v in (R - Rr).ravel()) < D("1e-50")
    eye = np.eye(m, dtype=np.int64).astype(object)
    assert max(abs(v) for v in (T - eye).ravel()) < D("1e-50")
    assert max(abs(v) for v in (W - Q @ R).ravel()) < D("1e-50")
    assert max(abs(v) for v in (S.T @ S - eye).ravel()) < D("1e-50")


def test_blas2_rgs_is_rhqr_of_zero_topped_matrix():
    """Section 6: RHQR of [0_m; W] with Psi = diag(I_m, Omega) gives u_j =
    [e_j; -q_j]: the same Q and R as BLAS2-RGS (up to the column signs of the
    reflector convention) and the same T."""
    n, m, k = 400, 8, 40
    W = ri.gaussian(n, m, 42)
    Om = np.random.default_rng(43).standard_normal((k, n)) / math.sqrt(k)
    Q, R, S, T = rhqr.blas2_rgs(W, Om)
    Wbar = np.concatenate([np.zeros((m, m)), W])
    skbar = sketch.ExplicitSketch(np.concatenate([np.zeros((k, m)), Om], axis=1))
    U, Sh, Th, Rh = rhqr.rhqr_left(Wbar, skbar)
    Qh = rhqr.form_q(U, Th)  # thin Q of [0; W]
    d = np.sign(np.diag(Rh)) * np.sign(np.diag(R))
    assert np.max(np.abs(Qh[:m])) <= 1e-13
    assert np.max(np.abs(Qh[m:] * d - Q)) <= 1e-12
    assert np.max(np.abs(d[:, None] * Rh - R)) <= 1e-12 * np.abs(R).max()
    assert np.max(np.abs(Th - T)) <= 1e-11


# ---------------------------------------------------------------------------
# trimRHQR (Section 7), right-looking
# ---------------------------------------------------------------------------


def _unit_first_columns(Om, m):
    Om = Om.copy()
    Om[:, :m] = Om[:, :m] / np.linalg.norm(Om[:, :m], axis=0)
    return Om


@pytest.mark.parametrize("scaling", ["unit", "norm"])
@pytest.mark.parametrize("k", [4, 12])  # fewer sampled rows than columns is allowed
def test_trim_rhqr_factorisation_and_elimination(scaling, k):
    n, m = 40, 6
    rng = np.random.default_rng(51)
    W = rng.standard_normal((n, m))
    Om = _unit_first_columns(rng.standard_normal((k, n)) / math.sqrt(k), m)
    U, S, beta, R = rhqr.trim_rhqr_right(W, Om, scaling)
    assert np.max(np.abs(S - Om @ U)) <= 1e-13
    assert np.allclose(np.tril(R, -1), 0)
    H = [rhqr.trim_reflector(U[:, j], Om, j, beta[j]) for j in range(m)]
    # the proposition: H_j leaves the first j entries and eliminates below j
    A = W.copy()
    for j in range(m):
        A = H[j] @ A
        assert np.max(np.abs(A[j + 1:, j])) <= 1e-12 * np.abs(W).max()
    # eq. trimrhqrfact: H_m ... H_1 W = [R; 0] and W = H_1 ... H_m [R; 0]
    assert np.max(np.abs(A[:m] - R)) <= 1e-12 * np.abs(R).max()
    P = np.eye(n)
    for j in range(m):
        P = P @ H[j]
    RW = np.zeros((n, m))
    RW[:m] = R
    assert np.max(np.abs(P @ RW - W)) <= 1e-12 * np.abs(W).max()
    # each H_j is sketch-isometric for Psi_j = diag(I_j, Omega_{j:n}) and an involution
    for j in range(m):
        Psi = np.zeros((j + k, n))
        Psi[:j, :j] = np.eye(j)
        Psi[j:, j:] = Om[:, j:]
        x = rng.standard_normal(n)
        assert abs(np.linalg.norm(Psi @ H[j] @ x) - np.linalg.norm(Psi @ x)) <= 1e-12 * np.linalg.norm(x)
        assert np.max(np.abs(H[j] @ H[j] - np.eye(n))) <= 1e-12
    # the diagonal of R: -sigma ||Omega w'|| at each step (unit-column Omega makes |r_jj| positive)
    assert np.all(np.abs(np.diag(R)) > 0)


@pytest.mark.parametrize("scaling", ["unit", "norm"])
def test_trim_rhqr_left_equals_right_and_compact_forms(scaling):
    n, m, k = 40, 6, 5  # fewer sampled rows than columns
    rng = np.random.default_rng(52)
    W = rng.standard_normal((n, m))
    Om = _unit_first_columns(rng.standard_normal((k, n)) / math.sqrt(k), m)
    Ur, Sr, br, Rr = rhqr.trim_rhqr_right(W, Om, scaling)
    U, S, T, Tt, R = rhqr.trim_rhqr_left(W, Om, scaling)
    assert np.max(np.abs(U - Ur)) <= 1e-12 and np.max(np.abs(S - Sr)) <= 1e-12
    assert np.max(np.abs(R - Rr)) <= 1e-12 * np.abs(R).max()
    # ut((Omega U)^t Omega) as a matrix, and the explicit reflectors
    L = np.stack([rhqr.trim_ut(S, Om, e) for e in np.eye(n)], axis=1)
    H = [rhqr.trim_reflector(U[:, j], Om, j, np.diag(T)[j]) for j in range(m)]
    right = np.eye(n)
    left = np.eye(n)
    for j in range(m):
        right = right @ H[j]
        left = H[j] @ left
    assert np.max(np.abs(right - (np.eye(n) - U @ T @ L))) <= 1e-12  # eq. compactrightbis
    assert np.max(np.abs(left - (np.eye(n) - U @ Tt.T @ L))) <= 1e-12  # eq. trimrhqrcompactfact
    # Woodbury forms (props woodburrybis and deltawoodburry)
    Ti = np.linalg.inv(T)
    assert np.max(np.abs(Ti + Ti.T - S.T @ S)) <= 1e-11
    assert np.max(np.abs(Tt.T + np.linalg.inv(Ti - L @ U))) <= 1e-10 * np.abs(Tt).max()
    # eq. trimrhqr_finalform
    RW = np.zeros((n, m))
    RW[:m] = R
    assert np.max(np.abs((np.eye(n) - U @ T @ L) @ RW - W)) <= 1e-12 * np.abs(W).max()
    assert np.max(np.abs((np.eye(n) - U @ Tt.T @ L) @ W - RW)) <= 1e-12 * np.abs(W).max()
