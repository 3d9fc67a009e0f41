"""Pin predicates for the FP64 oracle.

Each ``check_*`` runs one family of pins against the function(s) passed in and
returns the names of the pins that failed (empty list = pinned).  They are
parameterised by the functions under test so that ``test_oracle_mutants.py``
can feed deliberately broken variants (a flipped sign, a dropped term, a
transposed operand ...) and show that some pin catches each one.

What pins what (none of these re-types the oracle's own formula):
  * QR: hand-computed factorisations (tests/golden/qr_hand.json), the
    definition (Q^T Q = I, QR = Y, R upper triangular, diag(R) >= 0) and
    LAPACK's QR after the same sign normalisation.
  * SVD: closed forms (diagonal, rank one), a generator with a known spectrum,
    and LAPACK's SVD.
  * RU-QLP: exact recovery of exactly rank-k inputs (QQ^T A = A when
    range(A Omega) = range(A)), orthonormality / triangularity, the identity
    Q L P^T = Q Q^T A, the Eckart-Young lower bound (Section II-B-1), the
    deterministic bounds of Theorems 1, 2 and 5 with the actual Omega, the
    volume inequality prod_{i<=j} |L_ii| <= prod_{i<=j} sigma_i, and the
    transposition identity with the literal left-sketch Algorithm 1 + 2.
"""
from __future__ import annotations

import json
import os

import numpy as np

import paper_bounds as pb
from paper_2209_12464_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
SLACK = 1e-9


def _fail(fails, name, cond):
    if not cond:
        fails.append(name)


# ---------------------------------------------------------------------------
def check_qr(qr):
    fails = []
    with open(os.path.join(GOLDEN, "qr_hand.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        Q, R = qr(np.array(c["Y"]))
        _fail(fails, f"hand-{c['name']}-Q", np.allclose(Q, np.array(c["Q"]), atol=1e-15, rtol=0))
        _fail(fails, f"hand-{c['name']}-R", np.allclose(R, np.array(c["R"]), atol=1e-15, rtol=0))
    rng = np.random.default_rng(11)
    for (m, d) in [(50, 12), (7, 7), (300, 40)]:
        Y = rng.standard_normal((m, d)) * np.logspace(0, -6, d)[None, :]
        Q, R = qr(Y)
        _fail(fails, f"orth-{m}x{d}", np.linalg.norm(Q.T @ Q - np.eye(d)) < 1e-13)
        _fail(fails, f"backward-{m}x{d}", np.linalg.norm(Q @ R - Y) < 1e-14 * np.linalg.norm(Y))
        _fail(fails, f"triu-{m}x{d}", np.all(np.tril(R, -1) == 0.0))
        _fail(fails, f"diagpos-{m}x{d}", np.all(np.diag(R) >= 0.0))
        Ql, Rl = np.linalg.qr(Y)
        s = np.where(np.diag(Rl) < 0, -1.0, 1.0)
        _fail(fails, f"lapack-Q-{m}x{d}", np.allclose(Q, Ql * s[None, :], atol=1e-10, rtol=0))
        _fail(fails, f"lapack-R-{m}x{d}", np.allclose(R, Rl * s[:, None], atol=1e-12, rtol=1e-10))
    # rank deficient: a zero column and a repeated column
    Y = rng.standard_normal((20, 5))
    Y[:, 2] = 0.0
    Y[:, 4] = Y[:, 1]
    Q, R = qr(Y)
    _fail(fails, "rankdef-orth", np.linalg.norm(Q.T @ Q - np.eye(5)) < 1e-13)
    _fail(fails, "rankdef-backward", np.linalg.norm(Q @ R - Y) < 1e-14 * np.linalg.norm(Y))
    _fail(fails, "rankdef-zero-pivot", abs(R[2, 2]) < 1e-14 and abs(R[4, 4]) < 1e-13)
    return fails


# ---------------------------------------------------------------------------
def check_svd(svd):
    fails = []
    A = np.zeros((5, 3))
    A[0, 0], A[1, 1], A[2, 2] = 3.0, -1.0, 2.0
    _, s, _ = svd(A)
    _fail(fails, "diag", np.allclose(s, [3.0, 2.0, 1.0], atol=1e-15, rtol=0))
    u = np.array([1.0, 2.0, 2.0, 0.0])
    v = np.array([3.0, 0.0, 4.0])
    _, s, _ = svd(np.outer(u, v))
    _fail(fails, "rank1", abs(s[0] - 15.0) < 1e-13 and np.all(np.abs(s[1:]) < 1e-13))
    sig = np.geomspace(1.0, 1e-6, 12)
    A, _, _, _ = wl.dense_spectral(5, 30, 12, sig)
    U, s, V = svd(A)
    _fail(fails, "generator-spectrum", np.allclose(s, sig, atol=1e-14, rtol=0))
    _fail(fails, "reconstruct", np.linalg.norm(U @ np.diag(s) @ V.T - A) < 1e-13)
    _fail(fails, "V-orth", np.linalg.norm(V.T @ V - np.eye(12)) < 1e-13)
    B = np.random.default_rng(3).standard_normal((9, 14))
    _, s, _ = svd(B)
    _fail(fails, "lapack-wide", np.allclose(s, np.linalg.svd(B, compute_uv=False), atol=1e-13, rtol=0))
    return fails


# ---------------------------------------------------------------------------
def _bounds_case(ruqlp, sines, svd, n, k, p, q, sigma, seed):
    fails = []
    A, U, s, V = wl.dense_spectral(seed, n, n, sigma)
    Om = wl.omega(seed + 1, n, k + p)
    out = ruqlp(A, Om, q)
    Q, L, P = out["Q"], out["L"], out["P"]
    d = k + p
    tag = f"n{n}k{k}p{p}q{q}"
    w = pb.omega_ratio_norm(Om, V[:, :k])
    E = A - Q @ L @ P.T
    rF = np.linalg.norm(E)
    r2 = np.linalg.norm(E, 2)
    # Eckart-Young: rank-d approximation cannot beat the SVD tail.
    _fail(fails, f"eckart-young-2-{tag}", r2 >= s[d] * (1 - SLACK))
    _fail(fails, f"eckart-young-F-{tag}", rF >= np.sqrt(np.sum(s[d:] ** 2)) * (1 - SLACK))
    # Q L P^T = Q Q^T A  (B^T = A^T Q, P R_B = B^T)
    _fail(fails, f"QLP=QQtA-{tag}", np.linalg.norm(Q @ L @ P.T - Q @ (Q.T @ A)) < 1e-12 * np.linalg.norm(A))
    # Theorem 5 (both bounds), spectral and Frobenius norms.
    E2 = A - A @ P @ P.T
    for nm, val, bnd in [
        ("thm5-QQtA-2", r2, pb.thm5_QQtA(s, k, q, w, 2)),
        ("thm5-QQtA-F", rF, pb.thm5_QQtA(s, k, q, w, "F")),
        ("thm5-APPt-2", np.linalg.norm(E2, 2), pb.thm5_APPt(s, k, q, w, 2)),
        ("thm5-APPt-F", np.linalg.norm(E2), pb.thm5_APPt(s, k, q, w, "F")),
    ]:
        _fail(fails, f"{nm}-{tag}", val <= bnd * (1 + SLACK) + 1e-13)
    # Theorem 1 / Corollary 1 with roles swapped: L_11 = R_11^T, L_22 = R_22^T.
    # The leading k columns of Q (and so L_11) depend only on Omega[:, :k],
    # so the theorem is applied as its d = k instance (w_k); the paper's
    # lower bound on sigma_i(L_11) is replaced by the exact inequality
    # sigma_i(L_11) >= sigma_i cos(theta_max(Q_1, U_k)) plus Theorem 2's bound
    # on that angle (see test_paper_thm1_lower_bound_counterexample).
    wk = pb.omega_ratio_norm(Om[:, :k], V[:, :k])
    _, s11, _ = svd(L[:k, :k])
    _fail(fails, f"thm1-upper-{tag}", np.all(s11 <= s[:k] * (1 + SLACK)))
    sq1 = sines(Q[:, :k], U[:, :k])
    cmin = np.sqrt(max(0.0, 1.0 - sq1[-1] ** 2))
    _fail(fails, f"thm1-lower-{tag}", np.all(s11 >= s[:k] * cmin * (1 - SLACK)))
    _fail(fails, f"thm2-Q1-{tag}", np.all(sq1 <= pb.thm2_sin_Q(s, k, q, wk) * (1 + 1e-6) + 1e-14))
    _, s22, _ = svd(L[k:, k:])
    _fail(fails, f"thm1-L22-2-{tag}", s22[0] <= pb.thm1_upper_22(s, k, q, wk, 2) * (1 + SLACK) + 1e-13)
    _fail(fails, f"thm1-L22-F-{tag}",
          np.linalg.norm(L[k:, k:]) <= pb.thm1_upper_22(s, k, q, wk, "F") * (1 + SLACK) + 1e-13)
    # Theorem 2 with roles swapped: angle(P, V_k) ~ 2q+2, angle(Q, U_k) ~ 2q+1.
    sp = sines(P, V[:, :k])
    sq = sines(Q, U[:, :k])
    _fail(fails, f"thm2-P-{tag}", np.all(sp <= pb.thm2_sin_P(s, k, q, w) * (1 + 1e-6) + 1e-14))
    _fail(fails, f"thm2-Q-{tag}", np.all(sq <= pb.thm2_sin_Q(s, k, q, w) * (1 + 1e-6) + 1e-14))
    # volume inequality of the triangular factor
    dl = np.abs(np.diag(L))
    _fail(fails, f"volume-{tag}", np.all(np.cumsum(np.log(dl)) <= np.cumsum(np.log(s[:d])) + 1e-10))
    _fail(fails, f"L11<=sigma1-{tag}", dl[0] <= s[0] * (1 + SLACK))
    return fails


def check_ruqlp(ruqlp, paper, sines, svd, quick=False):
    fails = []
    # exact recovery on exactly rank-k inputs, d >= k
    for (m, n, k, p, q) in [(60, 50, 6, 4, 0), (45, 70, 5, 3, 1), (80, 40, 8, 0, 2)]:
        A, _, _, _ = wl.dense_spectral(100 + m, m, n, wl.spectrum_rank(min(m, n), k))
        Om = wl.omega(7 + n, n, k + p)
        out = ruqlp(A, Om, q)
        Q, L, P = out["Q"], out["L"], out["P"]
        d = k + p
        tag = f"{m}x{n}k{k}p{p}q{q}"
        rF = np.linalg.norm(A - Q @ L @ P.T) / np.linalg.norm(A)
        _fail(fails, f"exact-recovery-{tag}", rF <= 1e-13)
        _fail(fails, f"Q-orth-{tag}", np.linalg.norm(Q.T @ Q - np.eye(d)) < 1e-13)
        _fail(fails, f"P-orth-{tag}", np.linalg.norm(P.T @ P - np.eye(d)) < 1e-13)
        _fail(fails, f"L-lower-{tag}", np.all(np.triu(L, 1) == 0.0))
        _fail(fails, f"L-diagpos-{tag}", np.all(np.diag(L) >= 0.0))
        _fail(fails, f"shapes-{tag}", Q.shape == (m, d) and P.shape == (n, d) and L.shape == (d, d))
        # tail of diag(L) beyond the rank vanishes (rank revelation, Section III-A)
        if p > 0:
            _fail(fails, f"rank-reveal-{tag}", np.max(np.abs(np.diag(L)[k:])) < 1e-12)
    # deterministic bounds of Section IV on square gap / decay spectra
    cases = [(120, 8, 6, q, wl.spectrum_gap(120, 8, 0.1)) for q in (0, 1, 2)]
    cases += [(100, 10, 5, 1, wl.spectrum_decay(100, 10, 1))]
    if quick:
        cases = cases[1:2]
    for (n, k, p, q, sig) in cases:
        fails += _bounds_case(ruqlp, sines, svd, n, k, p, q, sig, seed=1000 + n + q)
    # transposition identity: right sketch of A == literal Algorithm 1 + 2 on A^T
    for (m, n, k, p, q) in [(70, 50, 6, 4, 1), (50, 90, 5, 5, 2), (40, 30, 4, 2, 0)]:
        A, _, _, _ = wl.dense_spectral(200 + m, m, n, wl.spectrum_gap(min(m, n), k, 0.05))
        Om = wl.omega(300 + n, n, k + p)
        out = ruqlp(A, Om, q, finish_paper=True)
        Qp, Pp, Lp, Rp = paper(A.T, Om, q)
        tag = f"{m}x{n}q{q}"
        _fail(fails, f"transpose-Q'=P-{tag}", np.allclose(Qp, out["P"], atol=1e-11, rtol=0))
        _fail(fails, f"transpose-R'=RB-{tag}", np.allclose(Rp, out["RB"], atol=1e-11, rtol=0))
        _fail(fails, f"transpose-L'=Rt^T-{tag}", np.allclose(Lp, out["Rtilde"].T, atol=1e-11, rtol=0))
        _fail(fails, f"transpose-P'=Qhat-{tag}", np.allclose(Pp, out["Qhat"], atol=1e-10, rtol=0))
    return fails


def check_csr(ruqlp):
    """CSR input gives the dense result (same algorithm, Section III-D)."""
    fails = []
    A = wl.csr_uniform(5, 90, 70, 0.15, planted_rank=4, planted_scale=3.0)
    D = wl.csr_to_dense(A)
    Om = wl.omega(6, 70, 10)
    a = ruqlp(A, Om, 1)
    b = ruqlp(D, Om, 1)
    for key in ("Q", "L", "P"):
        _fail(fails, f"csr-{key}", np.allclose(a[key], b[key], atol=1e-11, rtol=0))
    return fails
