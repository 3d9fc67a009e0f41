"""FP64 CPU oracle for Randomized Unpivoted QLP (RU-QLP), arXiv 2209.12464.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, call or execute this module; only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` leg (and its
``--impl reference`` arm) use it.  It shares no code with the CUDA path: its
inputs (A, Omega) come from the seeded generators and are passed in as arrays.

Everything is computed in IEEE float64 with plain numpy.  Library primitives
used as single steps: dense matrix products (numpy ``@``) and, for CSR inputs,
the sparse-times-dense product of ``scipy.sparse``.  The QR factorisation and
the SVD used by the pins are written out here (Householder reflections;
one-sided Jacobi), with no blocking, fusion or reordering.

Orientation.  The paper's Algorithm 1 (Section III-A) sketches from the left,
Phi in R^{m x d}, and orthonormalises A^T Phi.  This oracle runs the same
algorithm on the other side (Omega in R^{n x d}):

    Y = A Omega;  Q = orth(Y);  repeat q times {Z = A^T Q; Q~ = orth(Z);
    Y = A Q~; Q = orth(Y)};  B^T = A^T Q;  [P, R_B] = qr(B^T);  L = R_B^T,

so that A ~= Q L P^T = Q Q^T A.  This is Algorithm 1 + Algorithm 2 applied to
A^T with Phi = Omega, stopped before the d x d QR of R^T (Algorithm 1, step 5);
``ruqlp_paper`` is the literal left-sketch form, and ``ruqlp(...,
finish_paper=True)`` adds that d x d QR.  Tests check the two against each other.

Readings of the paper taken here (each also listed in the design notes):
  * orth() after every product of the power loop (Algorithm 2, Section III-B),
    not "once every few iterations";
  * the QR sign convention is diag(R) >= 0 (the paper states none); Householder
    vectors use v = x + sign(x_1)||x|| e_1 with sign(0) = +1;
  * q = 0 is allowed (Algorithm 1 without Algorithm 2).

Parity pins: every function here is pinned by ``tests/test_oracle_pins.py``
(hand examples, closed forms, library special cases, the paper's theorems).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "householder_qr", "orth", "jacobi_svd", "apply_A", "apply_At",
    "ruqlp", "ruqlp_paper", "residual_fro", "residual_fro_small",
    "spectral_norm", "principal_sines",
]


# ---------------------------------------------------------------------------
# Unpivoted QR (Section II-B-2: A = QR, Q orthonormal columns, R upper
# triangular).  Householder reflections, Golub & Van Loan Section 5.2.
# ---------------------------------------------------------------------------
def householder_qr(Y):
    """Thin unpivoted QR of a tall matrix, Y (m x d, m >= d) = Q R.

    Returns (Q, R): Q is m x d with orthonormal columns, R is d x d upper
    triangular with diag(R) >= 0.  Column j is reduced by the reflector
    H_j = I - beta_j v_j v_j^T with v_j = x + sign(x_1)||x|| e_1, which maps x
    to -sign(x_1)||x|| e_1; a zero column gives beta_j = 0 (H_j = I).  Q is
    formed explicitly as H_0 H_1 ... H_{d-1} [I_d; 0], and finally every
    column pair (Q_j, R_j.) with R_jj < 0 is negated.
    """
    W = np.array(Y, dtype=np.float64, copy=True)
    if W.ndim != 2:
        raise ValueError("householder_qr needs a 2-D array")
    m, d = W.shape
    if m < d:
        raise ValueError(f"householder_qr needs m >= d, got {m} x {d}")
    vs, betas = [], []
    for j in range(d):
        x = W[j:, j].copy()
        alpha = np.sqrt(np.dot(x, x))
        sgn = 1.0 if x[0] >= 0.0 else -1.0
        v = x
        v[0] = x[0] + sgn * alpha
        vtv = np.dot(v, v)
        beta = 0.0 if vtv == 0.0 else 2.0 / vtv
        if beta != 0.0:
            w = v @ W[j:, j:]
            W[j:, j:] -= beta * np.outer(v, w)
        vs.append(v)
        betas.append(beta)
    R = np.triu(W[:d, :])
    Q = np.zeros((m, d), dtype=np.float64)
    Q[:d, :d] = np.eye(d)
    for j in range(d - 1, -1, -1):
        if betas[j] != 0.0:
            v = vs[j]
            w = v @ Q[j:, :]
            Q[j:, :] -= betas[j] * np.outer(v, w)
    flip = np.where(np.diag(R) < 0.0, -1.0, 1.0)
    Q *= flip[None, :]
    R *= flip[:, None]
    return Q, R


def orth(Y):
    """orth() of Section II-A: an orthonormal basis of range(Y), taken as the Q
    factor of the unpivoted Householder QR above."""
    return householder_qr(Y)[0]


# ---------------------------------------------------------------------------
# One-sided Jacobi SVD (Hestenes 1958; Demmel & Veselic 1992), used as the
# brute-force singular values of tiny test matrices (Section II-B-1, Eq. (1)).
# ---------------------------------------------------------------------------
def jacobi_svd(A, tol=1e-15, max_sweeps=60):
    """SVD of a small dense matrix by one-sided Jacobi rotations.

    Rotates column pairs of W = A (A^T when m < n) until every pair is
    orthogonal to ``tol`` relative to the product of their norms; then
    sigma_i = ||w_i||, u_i = w_i / sigma_i, V = accumulated rotations.
    Returns (U, s, V) with s descending, A = U diag(s) V^T.
    """
    A = np.asarray(A, dtype=np.float64)
    transposed = A.shape[0] < A.shape[1]
    W = (A.T if transposed else A).copy()
    m, n = W.shape
    V = np.eye(n)
    for _ in range(max_sweeps):
        rotated = False
        for p in range(n - 1):
            for r in range(p + 1, n):
                alpha = np.dot(W[:, p], W[:, p])
                beta = np.dot(W[:, r], W[:, r])
                gamma = np.dot(W[:, p], W[:, r])
                if gamma == 0.0 or abs(gamma) <= tol * np.sqrt(alpha * beta):
                    continue
                rotated = True
                zeta = (beta - alpha) / (2.0 * gamma)
                t = (1.0 if zeta >= 0.0 else -1.0) / (abs(zeta) + np.sqrt(1.0 + zeta * zeta))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = c * t
                wp, wr = W[:, p].copy(), W[:, r].copy()
                W[:, p] = c * wp - s * wr
                W[:, r] = s * wp + c * wr
                vp, vr = V[:, p].copy(), V[:, r].copy()
                V[:, p] = c * vp - s * vr
                V[:, r] = s * vp + c * vr
        if not rotated:
            break
    sig = np.sqrt(np.sum(W * W, axis=0))
    order = np.argsort(-sig, kind="stable")
    sig = sig[order]
    W = W[:, order]
    V = V[:, order]
    U = np.zeros_like(W)
    nz = sig > 0.0
    U[:, nz] = W[:, nz] / sig[nz]
    if transposed:
        return V, sig, U
    return U, sig, V


# ---------------------------------------------------------------------------
# Products with A (dense or CSR): the O(mnd) / O(sd) steps (Section III-D).
# ---------------------------------------------------------------------------
def _as_operator(A):
    """Dense arrays become float64 ndarrays; CSR triples (rowptr, colidx,
    values, m, n) become a float64 scipy.sparse matrix."""
    if isinstance(A, dict):
        import scipy.sparse as sp
        return sp.csr_matrix(
            (np.asarray(A["values"], dtype=np.float64),
             np.asarray(A["colidx"], dtype=np.int64),
             np.asarray(A["rowptr"], dtype=np.int64)),
            shape=(int(A["m"]), int(A["n"])))
    return np.asarray(A, dtype=np.float64)


def _lowrank(A):
    """The (X, D, Y) of a low-rank term A = S + X D Y^T attached to a CSR dict
    under "lowrank" (float64), or None."""
    if isinstance(A, dict) and A.get("lowrank") is not None:
        lr = A["lowrank"]
        return tuple(np.asarray(lr[k], dtype=np.float64) for k in ("X", "D", "Y"))
    return None


def apply_A(A, X):
    """A X in float64 (sketch step Y = A Omega, Algorithm 1 step 3 / Section III-A).
    For A = S + X_l D Y_l^T: S X + X_l (D (Y_l^T X))."""
    X = np.asarray(X, dtype=np.float64)
    out = np.asarray(_as_operator(A) @ X)
    lr = _lowrank(A)
    if lr is not None:
        Xl, D, Yl = lr
        out = out + Xl @ (D @ (Yl.T @ X))
    return out


def apply_At(A, Y):
    """A^T Y in float64 (the transposed products of Algorithm 2 and B^T = A^T Q).
    For A = S + X_l D Y_l^T: S^T Y + Y_l (D^T (X_l^T Y))."""
    Y = np.asarray(Y, dtype=np.float64)
    out = np.asarray(_as_operator(A).T @ Y)
    lr = _lowrank(A)
    if lr is not None:
        Xl, D, Yl = lr
        out = out + Yl @ (D.T @ (Xl.T @ Y))
    return out


# ---------------------------------------------------------------------------
# RU-QLP (Algorithm 1 with Algorithm 2), right-sketch orientation.
# ---------------------------------------------------------------------------
def ruqlp(A, Omega, q, finish_paper=False):
    """RU-QLP of A with the Gaussian test matrix Omega (n x d) and q power steps.

    Steps (Section III-A, Algorithm 1 on A^T; Algorithm 2 for the power loop):
      Y = A Omega, Q = orth(Y);
      for i in 1..q: Z = A^T Q, Q~ = orth(Z), Y = A Q~, Q = orth(Y);
      B^T = A^T Q;  [P, R_B] = qr(B^T);  L = R_B^T.
    With ``finish_paper`` also [P~, R~] = qr(L) (Algorithm 1 step 5, the d x d
    QR of R^T in the paper's orientation), returning Qhat = Q P~ and R~, so that
    A ~= Qhat R~ P^T and diag(R~) are the paper's L-values of A^T.  With
    ``finish_paper=2`` (or "svd") instead the SVD of L (Section III-C, Remark
    1): Qsvd = Q U, Sigma, Psvd = P V with L = U diag(Sigma) V^T.

    A is a float64-convertible m x n array or a CSR dict (rowptr, colidx,
    values, m, n), optionally with a low-rank term "lowrank" = {X, D, Y}
    (A = S + X D Y^T, applied as products, never formed).  Returns a dict with Q (m x d), L (d x d lower triangular),
    P (n x d), RB (d x d) and, with finish_paper, Qhat and Rtilde.
    """
    Op = _as_operator(A)
    Omega = np.asarray(Omega, dtype=np.float64)
    m, n = Op.shape
    d = Omega.shape[1]
    if Omega.shape[0] != n:
        raise ValueError("Omega must be n x d")
    if not (1 <= d <= min(m, n)):
        raise ValueError("need 1 <= d <= min(m, n)")
    if q < 0:
        raise ValueError("q must be >= 0")
    Y = apply_A(A, Omega)
    Q = orth(Y)
    for _ in range(q):
        Z = apply_At(A, Q)
        Qt = orth(Z)
        Y = apply_A(A, Qt)
        Q = orth(Y)
    Bt = apply_At(A, Q)
    P, RB = householder_qr(Bt)
    out = {"Q": Q, "L": RB.T.copy(), "P": P, "RB": RB}
    if finish_paper == 2 or finish_paper == "svd":
        # Section III-C, Remark 1: L = U S V^T, A ~= (Q U) S (P V)^T
        U, sv, V = jacobi_svd(out["L"])
        out["Qsvd"] = Q @ U
        out["Sigma"] = sv
        out["Psvd"] = P @ V
    elif finish_paper:
        Pt, Rt = householder_qr(out["L"])
        out["Qhat"] = Q @ Pt
        out["Rtilde"] = Rt
    return out


def ruqlp_paper(A, Phi, q):
    """Literal Algorithm 1 (RU-QLP) with Algorithm 2 (PI_ORTH) for q >= 1.

    Phi is m x d.  Pbar = orth(A^T Phi); q times {B = A Pbar; Pbar = orth(B);
    B = A^T Pbar; Pbar = orth(B)}; [Q, R] = qr(A Pbar); [P~, R~] = qr(R^T);
    returns (Q, P = Pbar P~, L = R~^T, R).
    """
    A = np.asarray(A, dtype=np.float64)
    Phi = np.asarray(Phi, dtype=np.float64)
    Pbar = orth(A.T @ Phi)
    for _ in range(q):
        B = A @ Pbar
        Pbar = orth(B)
        B = A.T @ Pbar
        Pbar = orth(B)
    Q, R = householder_qr(A @ Pbar)
    Pt, Rt = householder_qr(R.T)
    return Q, Pbar @ Pt, Rt.T, R


# ---------------------------------------------------------------------------
# Measurements of a result (Section II-B-1 norms; Theorem 5 quantities).
# ---------------------------------------------------------------------------
def residual_fro_small(A, Q, L, P):
    """||A - Q L P^T||_F / ||A||_F formed explicitly (small dense A)."""
    A = np.asarray(A, dtype=np.float64)
    E = A - np.asarray(Q, np.float64) @ np.asarray(L, np.float64) @ np.asarray(P, np.float64).T
    return float(np.linalg.norm(E) / np.linalg.norm(A))


def residual_fro(A, Q, L, P):
    """||A - Q L P^T||_F / ||A||_F without forming an m x n product:
    ||A - M||^2 = ||A||^2 - 2 <A, M> + ||M||^2, M = Q L P^T, with
    <A, M> = sum((Q^T A P) * L) and ||M||^2 = sum((L^T (Q^T Q) L) * (P^T P)).
    Exact algebra; in float64 it resolves relative residuals down to ~1e-7.
    """
    Op = _as_operator(A)
    Q = np.asarray(Q, np.float64)
    L = np.asarray(L, np.float64)
    P = np.asarray(P, np.float64)
    if isinstance(Op, np.ndarray):
        a2 = float(np.sum(Op * Op))
    else:
        a2 = float(np.sum(Op.data * Op.data))
    lr = _lowrank(A)
    if lr is not None:
        # ||S + X D Y^T||^2 = ||S||^2 + 2 sum_{(i,j) in S} s_ij (X D Y^T)_ij
        #                     + trace(D^T (X^T X) D (Y^T Y))
        Xl, D, Yl = lr
        coo = Op.tocoo()
        XD = Xl @ D
        cross = 0.0
        for s0 in range(0, coo.nnz, 1 << 20):
            s1 = min(coo.nnz, s0 + (1 << 20))
            r, c = coo.row[s0:s1], coo.col[s0:s1]
            cross += float(np.sum(coo.data[s0:s1] * np.einsum("ij,ij->i", XD[r], Yl[c])))
        a2 = a2 + 2.0 * cross + float(np.trace(D.T @ (Xl.T @ Xl) @ D @ (Yl.T @ Yl)))
    QtAP = Q.T @ apply_A(A, P)
    am = float(np.sum(QtAP * L))
    m2 = float(np.sum((L.T @ (Q.T @ Q) @ L) * (P.T @ P)))
    r2 = max(a2 - 2.0 * am + m2, 0.0)
    return float(np.sqrt(r2 / a2))


def spectral_norm(matvec, rmatvec, n, iters=200, seed=0):
    """Largest singular value of a linear map by power iteration on M^T M."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n)
    x /= np.linalg.norm(x)
    s = 0.0
    for _ in range(iters):
        y = matvec(x)
        z = rmatvec(y)
        nz = np.linalg.norm(z)
        if nz == 0.0:
            return 0.0
        s = np.sqrt(nz)
        x = z / nz
    return float(s)


def principal_sines(X, W):
    """Sines of the k principal angles between range(X) (d columns) and
    range(W) (k <= d columns), both with orthonormal columns (Bjorck & Golub
    1973).  (I - W W^T) X has singular values sin(theta_1..k) and d - k ones,
    so the k smallest singular values of that projection are returned,
    ascending.  The projection form keeps tiny angles accurate (cosine form
    cannot resolve sines below ~1e-8)."""
    X = np.asarray(X, np.float64)
    W = np.asarray(W, np.float64)
    k = W.shape[1]
    S = X - W @ (W.T @ X)
    _, s, _ = jacobi_svd(S)
    return np.sort(s)[:k]
