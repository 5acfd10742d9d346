"""Randomized Householder QR, step by step in the paper's order (oracle side).

Indices are 0-based: the paper's column j (1..m) is ``j-1`` here.  Matrices
are numpy arrays; float64 arrays give the FP64 oracle, object arrays of
``decimal.Decimal`` give the same algorithm in extended precision (tests).

Readings of passages that are ambiguous or garbled:

* sign(0) := +1 in RHVector (Algorithm 2 is silent).
* Unit-diagonal scaling (Algorithm 2, second option) returns
  beta = 1 + |a|/rho = 2/||s||^2.  The printed "beta <- gamma/rho" is off by the
  sign sigma when a < 0; the appendix derives beta_u = 1 - a/rho for the
  unflipped vector, which is the same quantity.  The norm scaling
  (||s|| = sqrt 2) divides by sqrt(rho (rho + |a|)), again the sign-correct form.
* The T recurrence of Prop. "generalcompactwoodburry" uses beta_{j+1} in the new
  column (as in the deterministic recurrence of Section 2.2 and in
  Algorithm 4); the printed beta_j is a typo.
* Algorithm 6 writes ut(T^t Y^t Z) with Y = S_{1:m,1:m}, a dimension mismatch;
  the derivation in Section 3.3 uses the full S = Psi U, so M = ut(T^t S^t Z).
  Its "backward solve" of W_2 = X M runs forward over the columns (the explicit
  recursion of Section 3.3).
* The sketch step z <- RhSk(z) of Algorithm 7 is read as z <- RhSk(w) with w = A q_j.
* RHQR-GMRES uses beta e_1 := h_0 = (-sigma_1 rho_1) e_1 from the first
  reflector (Algorithm 8's sign<b,e_1>||c|| ignores x_0).
"""

from __future__ import annotations

import math

import numpy as np

from .sketch import rh_sketch


class Breakdown(ArithmeticError):
    """rho = 0 in RHVector: the trailing part of the column lies in Ker(Psi)
    (excluded by Prop. "elimination" and Thm. "mainthm")."""

    def __init__(self, column: int):
        super().__init__(f"randomized Householder breakdown at column {column}")
        self.column = column


def _sqrt(x):
    if hasattr(x, "sqrt"):
        return x.sqrt()
    return math.sqrt(x)


def _one(like):
    """1 in the arithmetic of array ``like``."""
    if like.dtype == object:
        return like.flat[0] * 0 + 1
    return 1.0


def _zeros(shape, like):
    z = np.zeros(shape, dtype=like.dtype)
    if like.dtype == object:
        z = z.astype(object) * _one(like) * 0
    return z


def _eye(m, like):
    e = _zeros((m, m), like)
    for i in range(m):
        e[i, i] = _one(like)
    return e


# ---------------------------------------------------------------------------
# Algorithm 2: RHVector
# ---------------------------------------------------------------------------


def rh_vector(w, y, j: int, scaling: str = "unit"):
    """Randomized Householder vector of column ``w`` with sketch ``y = Psi w`` at
    step ``j`` (Algorithm 2; elimination property eq. (sumup)).

    Returns u, s = Psi u, sigma, rho, beta with beta = 2/||s||^2, such that
    P(u, Psi) w = (w_{0:j}, -sigma rho, 0)."""
    a = y[j]
    sigma = -1 if a < 0 else 1
    s = _zeros(y.shape, y)
    s[j:] = y[j:]
    rho = _sqrt(np.sum(s[j:] * s[j:]))
    if rho == 0:
        raise Breakdown(j)
    u = _zeros(w.shape, w)
    u[j:] = w[j:]
    u[j] = u[j] + sigma * rho
    s[j] = s[j] + sigma * rho
    gamma = s[j]
    if scaling == "unit":  # <u, e_j> = 1
        u = u / gamma
        s = s / gamma
        beta = _one(y) + abs(a) / rho
    elif scaling == "norm":  # ||s|| = sqrt(2)
        f = _sqrt(rho * (rho + abs(a)))
        u = u / f
        s = s / f
        beta = _one(y)
    else:
        raise ValueError(scaling)
    return u, s, sigma, rho, beta


def t_column(T, S, s, beta, j: int):
    """New column of T (Prop. generalcompactwoodburry / Algorithm 4):
    t_j = (-beta T_{j-1} S_{j-1}^t s_j ; beta ; 0)."""
    col = _zeros((T.shape[0],), T)
    col[j] = beta
    if j > 0:
        col[:j] = -beta * (T[:j, :j] @ (S[:, :j].T @ s))
    return col


# ---------------------------------------------------------------------------
# Algorithm 3 (right-looking) and Algorithm 4 (left-looking)
# ---------------------------------------------------------------------------


def rhqr_right(W, sk, scaling: str = "unit"):
    """Algorithm 3.  Returns U, S, T, R (T built with the recurrence of
    Prop. generalcompactwoodburry, which Algorithm 3 does not form itself)."""
    W = np.array(W, copy=True)
    n, m = W.shape
    U = _zeros((n, m), W)
    S = _zeros((sk.k + m, m), W)
    T = _zeros((m, m), W)
    R = _zeros((m, m), W)
    for j in range(m):
        w = W[:, j].copy()
        YY = rh_sketch(W[:, j:], m, sk)  # [y Y] <- RhSk(W_{j:m})
        y, Y = YY[:, 0], YY[:, 1:]
        try:
            u, s, sigma, rho, beta = rh_vector(w, y, j, scaling)
        except Breakdown:
            raise
        R[:j, j] = w[:j]
        R[j, j] = -sigma * rho
        if j < m - 1:
            W[:, j + 1 :] = W[:, j + 1 :] - beta * np.outer(u, s @ Y)
        U[:, j] = u
        S[:, j] = s
        T[:, j] = t_column(T, S, s, beta, j)
    return U, S, T, R


def rhqr_left(W, sk, scaling: str = "unit"):
    """Algorithm 4 (left-looking RHQR).  Returns U, S, T, R with
    W = (I - U T S^t Psi)[R; 0] and Psi W = (I - S T S^t)[R; 0]."""
    W = np.asarray(W)
    n, m = W.shape
    U = _zeros((n, m), W)
    S = _zeros((sk.k + m, m), W)
    T = _zeros((m, m), W)
    R = _zeros((m, m), W)
    for j in range(m):
        w = W[:, j].copy()
        y = rh_sketch(w, m, sk)
        if j >= 1:
            c = T[:j, :j].T @ (S[:, :j].T @ y)
            w = w - U[:, :j] @ c  # refresh w_j with the previous reflectors
            y = rh_sketch(w, m, sk)
        u, s, sigma, rho, beta = rh_vector(w, y, j, scaling)
        R[:j, j] = w[:j]
        R[j, j] = -sigma * rho
        T[:, j] = t_column(T, S, s, beta, j)
        U[:, j] = u
        S[:, j] = s
    return U, S, T, R


def block_rhqr(W, sk, bs: int, scaling: str = "unit"):
    """Algorithm 5 (blockRHQR): the columns of W in blocks of `bs`; block j is
    first refreshed with the reflectors of every earlier block, one block at a
    time (W^(j) <- W^(j) - U^(k) T^(k)t S^(k)t Psi W^(j), k < j: the printed
    inner loop writes U^(j) where the earlier block U^(k) is meant), its rows
    above the block give R's off-diagonal block, and Algorithm 4 factors it with
    the global Psi = diag(I_m, Omega) and the global column indices.  Returns R
    and the list of (first column, U^(j), S^(j), T^(j)).  In exact arithmetic
    the reflectors are those of Algorithm 4 on the whole W and T^(j) is the
    diagonal block of its T."""
    W = np.asarray(W)
    n, m = W.shape
    R = _zeros((m, m), W)
    blocks = []
    for c0 in range(0, m, bs):
        c1 = min(m, c0 + bs)
        Wj = W[:, c0:c1].copy()
        for _, Uk, Sk, Tk in blocks:
            Y = rh_sketch(Wj, m, sk)
            Wj = Wj - Uk @ (Tk.T @ (Sk.T @ Y))
        R[:c0, c0:c1] = Wj[:c0]
        b = c1 - c0
        U = _zeros((n, b), W)
        S = _zeros((sk.k + m, b), W)
        T = _zeros((b, b), W)
        for i in range(b):
            j = c0 + i  # global column
            w = Wj[:, i].copy()
            if i >= 1:
                y = rh_sketch(w, m, sk)
                c = T[:i, :i].T @ (S[:, :i].T @ y)
                w = w - U[:, :i] @ c
            y = rh_sketch(w, m, sk)
            u, sv, sigma, rho, beta = rh_vector(w, y, j, scaling)
            R[c0:j, j] = w[c0:j]
            R[j, j] = -sigma * rho
            T[:, i] = t_column(T, S, sv, beta, i)
            U[:, i] = u
            S[:, i] = sv
        blocks.append((c0, U, S, T))
    return R, blocks


def trim_rhqr_right(W, Omega, scaling: str = "unit"):
    """Right-looking trimRHQR (Section 7, Algorithms 10-11) with the reflectors
    H(u_j, Omega, j) = I - beta u_j (Omega u_j)^t [0 Omega_{j:n}] of eq. rhousebisbis.
    Omega (l x n) must have unit first m columns.  Column j: w' = (0_j; w_{j:}),
    rho = ||Omega w'||, sigma = sign(w_j) (sign(0) = +1), v = w' + sigma rho e_j,
    s = Omega v, then either u = v / v_j (unit diagonal, beta = 2/||s||^2) or
    u = sqrt(2) v / ||s|| (beta = 1); r_{0:j} = w_{0:j}, r_jj = -sigma rho; the
    trailing columns get H(u, Omega, j).  (Readings: the scale alpha is the
    reciprocal of v's first entry, as for Algorithm 2, rather than "the first
    entry of v'", and the trailing update runs for every j, not only j >= 2.)
    Returns U, S = Omega U, beta, R with W = H_1 ... H_m [R; 0]."""
    W = np.array(W, copy=True)
    n, m = W.shape
    U = _zeros((n, m), W)
    S = _zeros((Omega.shape[0], m), W)
    R = _zeros((m, m), W)
    beta = _zeros((m,), W)
    for j in range(m):
        w = W[:, j].copy()
        wp = w.copy()
        wp[:j] = 0 * wp[:j]
        z = Omega @ wp
        rho = _sqrt(z @ z)
        if rho == 0:
            raise Breakdown(j)
        sigma = -1 if w[j] < 0 else 1
        v = wp.copy()
        v[j] = v[j] + sigma * rho
        sv = Omega @ v
        if scaling == "unit":
            g = v[j]
            u, sv = v / g, sv / g
            b = 2 / (sv @ sv)
        else:
            a = _sqrt(2 * _one(W)) / _sqrt(sv @ sv)
            u, sv = v * a, sv * a
            b = _one(W)
        R[:j, j] = w[:j]
        R[j, j] = -sigma * rho
        if j < m - 1:
            X = Omega[:, j:] @ W[j:, j + 1:]
            W[:, j + 1:] = W[:, j + 1:] - b * np.outer(u, sv @ X)
        U[:, j], S[:, j], beta[j] = u, sv, b
    return U, S, beta, R


def trim_ut(S, Omega, x):
    """ut((Omega U)^t Omega) x: entry i is s_i . (Omega_{i:n} x_{i:n}) (row i of the
    product with the columns before i removed), S = Omega U."""
    out = _zeros((S.shape[1],) + x.shape[1:], x)
    for i in range(S.shape[1]):
        out[i] = S[:, i] @ (Omega[:, i:] @ x[i:])
    return out


def trim_rhqr_left(W, Omega, scaling: str = "unit"):
    """Left-looking trimRHQR (Section 7): column j is refreshed with the earlier
    reflectors through the compact left-wise form H_{j-1} ... H_1 = I - U Tt^t
    ut((Omega U)^t Omega) (eq. trimrhqrcompactfact), then trimRHVector gives u_j.
    T (right-wise compositions, the recurrence of eq. Tqdefbis) and Tt (left-wise,
    eq. Sqdefbis) take t_{0:j,j} = -beta_j T_{0:j,0:j} S_{0:j}^t s_j and
    tt_{0:j,j} = -beta_j Tt_{0:j,0:j} ([0 Omega_{j:n}] U_{0:j})^t s_j, diagonals beta_j.
    Returns U, S = Omega U, T, Tt, R (eq. trimrhqr_finalform)."""
    W = np.asarray(W)
    n, m = W.shape
    U = _zeros((n, m), W)
    S = _zeros((Omega.shape[0], m), W)
    T = _zeros((m, m), W)
    Tt = _zeros((m, m), W)
    R = _zeros((m, m), W)
    for j in range(m):
        w = W[:, j].copy()
        if j:
            w = w - U[:, :j] @ (Tt[:j, :j].T @ trim_ut(S[:, :j], Omega, w))
        wp = w.copy()
        wp[:j] = 0 * wp[:j]
        z = Omega @ wp
        rho = _sqrt(z @ z)
        if rho == 0:
            raise Breakdown(j)
        sigma = -1 if w[j] < 0 else 1
        v = wp.copy()
        v[j] = v[j] + sigma * rho
        sv = Omega @ v
        if scaling == "unit":
            g = v[j]
            u, sv = v / g, sv / g
            b = 2 / (sv @ sv)
        else:
            a = _sqrt(2 * _one(W)) / _sqrt(sv @ sv)
            u, sv = v * a, sv * a
            b = _one(W)
        R[:j, j] = w[:j]
        R[j, j] = -sigma * rho
        if j:
            T[:j, j] = -b * (T[:j, :j] @ (S[:, :j].T @ sv))
            OU = Omega[:, j:] @ U[j:, :j]  # [0 Omega_{j:n}] U_{0:j}
            Tt[:j, j] = -b * (Tt[:j, :j] @ (OU.T @ sv))
        T[j, j] = b
        Tt[j, j] = b
        U[:, j], S[:, j] = u, sv
    return U, S, T, Tt, R


def trim_reflector(u, Omega, j: int, beta):
    """Explicit H(u, Omega, j) = I - beta u (Omega u)^t [0_{l x j} Omega_{j:n}] (small n only)."""
    n = u.shape[0]
    Om = Omega.copy()
    Om[:, :j] = 0 * Om[:, :j]
    return np.eye(n) - beta * np.outer(u, (Omega @ u) @ Om)


def rgs(W, Omega):
    """Randomized Gram-Schmidt with a given Omega (k x n): r = (Omega Q)^t Omega w_j
    (the sketched least-squares coefficients, Omega Q having orthonormal
    columns), q~ = w_j - Q r, R_jj = ||Omega q~||, q_j = q~ / R_jj.  The
    reference that BLAS2-RGS (Section 6) equals in exact arithmetic."""
    W = np.asarray(W)
    n, m = W.shape
    Q = _zeros((n, m), W)
    R = _zeros((m, m), W)
    SQ = _zeros((Omega.shape[0], m), W)  # Omega Q
    for j in range(m):
        w = W[:, j].copy()
        if j:
            r = SQ[:, :j].T @ (Omega @ w)
            w = w - Q[:, :j] @ r
            R[:j, j] = r
        z = Omega @ w
        rho = _sqrt(z @ z)
        R[j, j] = rho
        Q[:, j] = w / rho
        SQ[:, j] = z / rho
    return Q, R


def blas2_rgs(W, Omega):
    """Algorithm 9 (BLAS2-RGS): RHQR of [0_m; W] written on W (Section 6).
    Column j: z = Omega w_j, r = T_{j-1}^t S_{j-1}^t z, w = w_j - Q_{j-1} r,
    z = Omega w, rho = ||z||, q_j = w / rho, s_j = z / rho, R[:j, j] = r,
    R_jj = rho, T[:j, j] = -T_{j-1} S_{j-1}^t s_j, T_jj = 1.  (The printed
    rho = ||Omega z|| and s_j = rho^{-1} s are read as ||z|| and z / rho, as
    the derivation before it gives.)  Returns Q, R, S = Omega Q and T, which
    equals I in exact arithmetic and records the loss of sketched
    orthogonality in floating point."""
    W = np.asarray(W)
    n, m = W.shape
    Q = _zeros((n, m), W)
    R = _zeros((m, m), W)
    S = _zeros((Omega.shape[0], m), W)
    T = _zeros((m, m), W)
    for j in range(m):
        w = W[:, j].copy()
        if j:
            r = T[:j, :j].T @ (S[:, :j].T @ (Omega @ w))
            w = w - Q[:, :j] @ r
            R[:j, j] = r
        z = Omega @ w
        rho = _sqrt(z @ z)
        R[j, j] = rho
        Q[:, j] = w / rho
        S[:, j] = z / rho
        if j:
            T[:j, j] = -(T[:j, :j] @ (S[:, :j].T @ S[:, j]))
        T[j, j] = _one(T)
    return Q, R, S, T


def form_q(U, T, m: int | None = None):
    """Thin Q factor Q = [I_m; 0] - U T U_{1:m,1:m}^t (Section 3.2)."""
    n, mm = U.shape
    m = mm if m is None else m
    Q = -(U @ (T @ U[:m, :].T))
    for i in range(m):
        Q[i, i] = Q[i, i] + _one(U)
    return Q


def compact_apply(U, T, S, sk, X, m: int, transpose: bool = False):
    """(I - U T S^t Psi) X, or with T^t (eq. generalcompact)."""
    TT = T.T if transpose else T
    return X - U @ (TT @ (S.T @ rh_sketch(X, m, sk)))


def householder_qr(Z, scaling: str = "unit"):
    """Deterministic Householder QR of Z (p x m, p >= m) in the conventions of
    Algorithm 2 with Psi = I: returns the Householder vectors S, the T factor of
    the recurrence in Section 2.2 and R, with Z = (I - S T S^t)[R; 0]."""
    Z = np.array(Z, copy=True)
    p, m = Z.shape
    S = _zeros((p, m), Z)
    T = _zeros((m, m), Z)
    R = _zeros((m, m), Z)
    for j in range(m):
        z = Z[:, j].copy()
        a = z[j]
        sigma = -1 if a < 0 else 1
        rho = _sqrt(np.sum(z[j:] * z[j:]))
        if rho == 0:
            raise Breakdown(j)
        v = _zeros((p,), Z)
        v[j:] = z[j:]
        v[j] = v[j] + sigma * rho
        if scaling == "unit":
            gamma = v[j]
            v = v / gamma
            beta = _one(Z) + abs(a) / rho
        else:
            v = v / _sqrt(rho * (rho + abs(a)))
            beta = _one(Z)
        R[:j, j] = z[:j]
        R[j, j] = -sigma * rho
        if j < m - 1:  # apply P(v) = I - beta v v^t to the trailing columns
            Z[:, j + 1 :] = Z[:, j + 1 :] - beta * np.outer(v, v @ Z[:, j + 1 :])
        S[:, j] = v
        T[:, j] = t_column(T, S, v, beta, j)
    return S, T, R


# ---------------------------------------------------------------------------
# Algorithm 6: recRHQR, and refinement passes
# ---------------------------------------------------------------------------


def rec_rhqr(W, sk, scaling: str = "unit"):
    """Algorithm 6.  Z = Psi W; (S, T, R) = HQR(Z); U_1 = S_{1:m};
    M = ut(T^t S^t Z); U_2 solves W_2 = U_2 M by the column recursion
    x_j = (w_j - sum_{i<j} x_i M_ij) / M_jj (Section 3.3).
    Returns U, S, T, R, M."""
    W = np.asarray(W)
    n, m = W.shape
    Z = rh_sketch(W, m, sk)
    S, T, R = householder_qr(Z, scaling)
    Y = S[:m, :]
    M = np.triu(T.T @ (S.T @ Z))
    W2 = W[m:, :]
    X = _zeros(W2.shape, W)
    for j in range(m):
        acc = W2[:, j] - X[:, :j] @ M[:j, j] if j else W2[:, j].copy()
        X[:, j] = acc / M[j, j]
    U = np.concatenate([Y, X], axis=0)
    return U, S, T, R, M


def rec_rhqr_refined(W, sk, passes: int = 2, scaling: str = "unit"):
    """recRHQR repeated on its own Q factor: X_0 = W, (U_i, S_i, T_i, R_i) =
    recRHQR(X_{i-1}), X_i = Q(U_i, T_i), R = R_p ... R_1.

    The last pass's (U, S, T) represent the final Q as a product of randomized
    reflectors, and P_m ... P_1 W = [R; 0], so (U, S, T, R) is a randomized
    Householder factorization of W.  Returns Q, R, U, S, T."""
    W = np.asarray(W)
    m = W.shape[1]
    X = W
    Racc = _eye(m, W)
    out = None
    for _ in range(passes):
        U, S, T, R, _M = rec_rhqr(X, sk, scaling)
        X = form_q(U, T, m)
        Racc = R @ Racc
        out = (U, S, T)
    return (X, Racc) + out


def lu_reconstruct(Q, sk):
    """Eq. (sketchedlufact): [I_m; 0] - Psi Q = S (T U_1^t) is the unique LU
    factorisation with unit lower-triangular S.  Returns U, S, T with
    U_1 = S_{1:m}, T = G U_1^{-t} and U_2 = -Q_2 G^{-1}, G = T U_1^t."""
    n, m = Q.shape
    B = -rh_sketch(Q, m, sk)
    for i in range(m):
        B[i, i] = B[i, i] + _one(Q)
    p = B.shape[0]
    L = _zeros((p, m), Q)
    G = _zeros((m, m), Q)
    A = B.copy()
    for j in range(m):  # Doolittle elimination without pivoting
        G[j, j:] = A[j, j:]
        L[j, j] = _one(Q)
        L[j + 1 :, j] = A[j + 1 :, j] / A[j, j]
        A[j + 1 :, j + 1 :] = A[j + 1 :, j + 1 :] - np.outer(L[j + 1 :, j], G[j, j + 1 :])
    S = L
    U1 = S[:m, :]
    T = solve_upper_right(G, U1.T)  # T U_1^t = G
    U2 = -solve_upper_right(Q[m:, :], G)  # U_2 G = -Q_2
    return np.concatenate([U1, U2], axis=0), S, T


def solve_upper_right(B, A):
    """X with X A = B for upper-triangular A (forward over the columns)."""
    X = _zeros(B.shape, B)
    m = A.shape[0]
    for j in range(m):
        acc = B[:, j] - X[:, :j] @ A[:j, j] if j else B[:, j].copy()
        X[:, j] = acc / A[j, j]
    return X


# ---------------------------------------------------------------------------
# Algorithm 7 (RHQR-Arnoldi) and Algorithm 8 (RHQR-GMRES)
# ---------------------------------------------------------------------------


class RHQRArnoldi:
    """Algorithm 7 with Psi = diag(I_{mmax+1}, Omega): the Krylov basis is kept in
    the compact form (U, S, T) of its mmax+1 randomized reflectors."""

    def __init__(self, sk, n: int, mmax: int, scaling: str = "unit", like=None):
        like = np.zeros(1) if like is None else like
        self.sk, self.n, self.mmax, self.scaling = sk, n, mmax, scaling
        self.M = mmax + 1
        self.U = _zeros((n, self.M), like)
        self.S = _zeros((sk.k + self.M, self.M), like)
        self.T = _zeros((self.M, self.M), like)
        self.j = 0

    def psi(self, x):
        return rh_sketch(x, self.M, self.sk)

    def _reflect(self, w, z):
        """Reflector j of (w, z = Psi w): h_{j-1} = (w_{0:j}, -sigma rho, 0)."""
        j = self.j
        u, s, sigma, rho, beta = rh_vector(w, z, j, self.scaling)
        h = _zeros((self.M,), self.T)
        h[:j] = w[:j]
        h[j] = -sigma * rho
        self.T[:, j] = t_column(self.T, self.S, s, beta, j)
        self.U[:, j] = u
        self.S[:, j] = s
        self.j += 1
        return h

    def basis_vector(self, j: int):
        """q_j = e_j - U_j T_j S_j^t e_j (0-based j, uses reflectors 0..j)."""
        J = j + 1
        q = -(self.U[:, :J] @ (self.T[:J, :J] @ self.S[j, :J]))
        q[j] = q[j] + _one(self.T)
        return q

    def begin(self, r0):
        """First reflector from r0 = b - A x0; returns h_0 and q_1."""
        h0 = self._reflect(r0, self.psi(r0))
        return h0, self.basis_vector(0)

    def step(self, Aq):
        """Given w = A q_j for the newest basis vector, refresh it with the
        reflectors so far, take the next reflector and return (h_j, q_{j+1})."""
        J = self.j
        z = self.psi(Aq)
        w = Aq - self.U[:, :J] @ (self.T[:J, :J].T @ (self.S[:, :J].T @ z))
        z = self.psi(w)
        h = self._reflect(w, z)
        q = self.basis_vector(J) if J < self.M else None
        return h, q


def rhqr_arnoldi(A, b, x0, sk, mmax: int, scaling: str = "unit"):
    """Algorithm 7 driver.  Returns H (mmax+1 x mmax), the explicit basis
    Q (n x (mmax+1)), h_0 and the Arnoldi object (compact U, S, T)."""
    n = b.shape[0]
    arn = RHQRArnoldi(sk, n, mmax, scaling, like=np.asarray(b))
    h0, q = arn.begin(b - A(x0))
    Q = [q]
    H = _zeros((mmax + 1, mmax), np.asarray(b))
    for j in range(mmax):
        h, q = arn.step(A(Q[-1]))
        H[:, j] = h
        Q.append(q)
    return H, np.stack(Q, axis=1), h0, arn


def rhqr_gmres(A, b, x0, sk, mmax: int, scaling: str = "unit"):
    """Algorithm 8 (one cycle): x = x0 + Q_m y with
    y = argmin || h_0 - H y ||  (eq. rgmresopti).  float64 only."""
    H, Q, h0, _ = rhqr_arnoldi(A, b, x0, sk, mmax, scaling)
    y = np.linalg.lstsq(H, h0, rcond=None)[0]
    return x0 + Q[:, :mmax] @ y, H, Q, h0
