"""Exactly rank-deficient sketches and the Householder-TSQR orth() (Section
II-A's unpivoted QR), through the C ABI.

An exactly rank-k A with d = k + p > k makes every sketch of rank k: its
trailing d - k directions are rounding noise.  Shifted CholeskyQR3 often still
returns an orthonormal Q there (its passes normalise the noise directions, as
Householder QR does); when it cannot, the last pass meets a Gram far from I,
flags RUQLP_FLAG_RANKDEF and the library redoes the decomposition with TSQR
(RUQLP_FLAG_TSQR).  Either way the result must satisfy what is unique, checked
against the FP64 oracle on the same values (its own Householder QR):

  * the leading k columns of Q and P and the leading k columns of L (the first
    k rows of R_B): element-wise, the FP64 / FP32 tolerances of the dense
    parity test.  On the BF16 path the sketches' operands are rounded to
    BF16, which moves the basis inside range(A) by ~2^-9, so there the
    unique quantities are the span of Q's leading k columns (range(A)) and
    the singular values of L's leading k x k block (those of A);
  * exact recovery: the relative residual ||A - Q L P^T||_F / ||A||_F is at
    rounding level (1e-12 FP64, 2e-5 FP32, 5e-5 BF16) and range(A) lies in
    range(Q);
  * |L_ii| <= tol |L_11| for i > k (the rank is revealed), Q and P orthonormal.

A is X Y^T with X, Y of entries in {-1, 0, 1}: integers of magnitude <= k, so
it is exact (and exactly rank k) in FP64, FP32 and BF16 alike.  TSQR is also
checked on full-rank inputs (option orth_tsqr) element-wise against the
oracle, as a QR in its own right.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_12464_gb300 import ruqlp
from paper_2209_12464_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

DT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}
TOLL = {"f64": 1e-10, "f32": 1e-5, "bf16": 1e-3}
TOLQ = {"f64": 1e-9, "f32": 1e-4, "bf16": 1e-3}
TOLR = {"f64": 1e-12, "f32": 2e-5, "bf16": 5e-5}
TOLO = {"f64": 1e-12, "f32": 2e-5, "bf16": 2e-5}


@pytest.fixture(scope="module")
def handle():
    import __graft_entry__ as g
    g.build()
    h = ruqlp.Handle(0, torch.cuda.current_stream().cuda_stream)
    yield h
    h.close()


def _rank_k(seed, m, n, k):
    rng = np.random.default_rng(seed)
    X = rng.integers(-1, 2, size=(m, k)).astype(np.float64)
    Y = rng.integers(-1, 2, size=(n, k)).astype(np.float64)
    return X @ Y.T


# m, n, k, p, q: small, m < n, q = 0 and 2, a tall sketch (tensor-core Gram /
# Q = Y R^-1 on the CholeskyQR attempt), one past the blocked Cholesky
RANK_CASES = [(600, 400, 12, 8, 1), (300, 700, 10, 6, 0), (900, 800, 20, 12, 2),
              (9000, 1200, 40, 24, 1), (1200, 1000, 280, 20, 1)]


# cases where the CholeskyQR attempt is known to flag the sketch (the
# automatic TSQR rerun is taken): d = 300, past the blocked Cholesky
FALLBACK_CASES = {(1200, 1000, 280, 20, 1)}


@pytest.mark.parametrize("orth", ["auto", "tsqr"])
@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("case", RANK_CASES, ids=[f"{a}x{b}k{c}p{d}q{e}" for a, b, c, d, e in RANK_CASES])
def test_exact_rank_k_recovered(handle, case, dt, orth):
    """auto: CholeskyQR, with the TSQR rerun if it flags the sketch (and
    always on the FALLBACK_CASES); tsqr: option orth_tsqr, every orth() a
    Householder TSQR."""
    m, n, k, p, q = case
    if dt == "bf16" and k > 200:
        pytest.skip("integer entries up to k must stay exact in BF16 (|a| <= 256)")
    d = k + p
    A = _rank_k(m + 7 * n + k, m, n, k)
    Om = wl.omega(m + n + q, n, d)
    Ag = wl.aligned_rows(torch.from_numpy(A).to(DT[dt]).cuda())
    assert np.array_equal(Ag.double().cpu().numpy(), A)
    handle.set_option("orth_tsqr", 1 if orth == "tsqr" else 0)
    try:
        Q, L, P, flags = handle.decompose(Ag, torch.from_numpy(Om).cuda(), k, p, q)
    finally:
        handle.set_option("orth_tsqr", 0)
    if orth == "tsqr":
        assert flags & ruqlp.FLAG_TSQR, flags
    elif flags & ruqlp.FLAG_RANKDEF or case in FALLBACK_CASES:
        assert flags & ruqlp.FLAG_RANKDEF and flags & ruqlp.FLAG_TSQR, flags
    else:
        assert flags & ruqlp.FLAG_TSQR == 0, flags
    Q, L, P = (t.double().cpu().numpy() for t in (Q, L, P))
    ref = oracle.ruqlp(A, Om, q)
    l11 = abs(ref["L"][0, 0])
    assert np.all(np.triu(L, 1) == 0.0)
    assert np.max(np.abs(Q.T @ Q - np.eye(d))) <= TOLO[dt] * max(1.0, d / 64)
    assert np.max(np.abs(P.T @ P - np.eye(d))) <= TOLO[dt] * max(1.0, d / 64)
    if dt != "bf16":
        assert np.max(np.abs(Q[:, :k] - ref["Q"][:, :k])) <= TOLQ[dt]
        assert np.max(np.abs(P[:, :k] - ref["P"][:, :k])) <= TOLQ[dt]
        assert np.max(np.abs(L[:, :k] - ref["L"][:, :k])) <= TOLL[dt] * l11
    assert np.max(np.abs(np.diag(L)[k:])) <= max(TOLL[dt], 1e-6) * l11
    r = oracle.residual_fro_small(A, Q, L, P)
    assert r <= TOLR[dt], r
    U, sa, _ = np.linalg.svd(A, full_matrices=False)
    U = U[:, :k]
    Qk = Q[:, :k]
    assert np.linalg.norm(U - Qk @ (Qk.T @ U), 2) <= 10 * TOLQ[dt]
    sl = np.linalg.svd(L[:k, :k], compute_uv=False)
    assert np.max(np.abs(sl - sa[:k])) <= 10 * TOLL[dt] * sa[0]


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_full_rank_input_takes_no_fallback(handle, dt):
    """The dense workload form (gap then 1e-2 / (i - k), small noise): no
    RUQLP_FLAG_RANKDEF, so no TSQR rerun."""
    m, n, k, p, q = 2000, 1500, 60, 20, 2
    A, _, _, _ = wl.dense_spectral(5, m, n, wl.spectrum_gap(n, k, 1e-2), noise_std=1e-6)
    Om = wl.omega(6, n, k + p)
    Q, L, P, flags = handle.decompose(torch.from_numpy(A).to(DT[dt]).cuda(),
                                      torch.from_numpy(Om).cuda(), k, p, q)
    assert flags & (ruqlp.FLAG_RANKDEF | ruqlp.FLAG_TSQR) == 0, flags


ORTH_RANK = [(1000, 30, 10), (20011, 220, 150), (6000, 300, 200), (4000, 170, 100)]


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("case", ORTH_RANK, ids=[f"{a}x{b}r{c}" for a, b, c in ORTH_RANK])
def test_orth_entry_rank_deficient_y(handle, case, dt):
    """ruqlp_orth of an exactly rank-r Y (r < d): orthonormal Q whose leading
    r columns equal the oracle's Householder Q (Y's first r columns are
    independent) and whose span holds range(Y).  Covers TSQR leaves and tree
    nodes in shared memory and in global memory (d = 300 FP32, d >= 160 FP64)."""
    M, d, r = case
    rng = np.random.default_rng(M + d + r)
    Y = rng.standard_normal((M, r)) @ rng.standard_normal((r, d))
    Yg = torch.from_numpy(Y).to(DT[dt]).cuda()
    Yh = Yg.double().cpu().numpy()
    Q = handle.orth(Yg).double().cpu().numpy()
    Qr, _ = oracle.householder_qr(Yh)
    u = 2.0 ** -53 if dt == "f64" else 2.0 ** -24
    assert np.max(np.abs(Q.T @ Q - np.eye(d))) <= 50 * d * u
    kap = np.linalg.cond(Yh[:, :r])
    assert np.max(np.abs(Q[:, :r] - Qr[:, :r])) <= 50 * kap * u * max(1.0, np.sqrt(d))
    Uy = np.linalg.svd(Yh, full_matrices=False)[0][:, :r]
    assert np.linalg.norm(Uy - Q @ (Q.T @ Uy), 2) <= 100 * kap * u * np.sqrt(d)


TSQR_FULL = [(1000, 30, 1), (20011, 220, 3), (5003, 64, 6), (300, 300, 2), (129, 1, 0),
             (6000, 300, 2), (4000, 170, 3), (150000, 64, 2)]


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("case", TSQR_FULL, ids=[f"{a}x{b}k1e{c}" for a, b, c in TSQR_FULL])
def test_tsqr_orth_matches_householder_q(handle, case, dt):
    """Option orth_tsqr: ruqlp_orth as a Householder TSQR, element-wise
    against the oracle's Householder Q (the bound of the CholeskyQR test:
    50 kappa u sqrt(d)); orthonormal to 50 d u whatever kappa."""
    M, d, lk = case
    rng = np.random.default_rng(M + d + lk)
    Y = (wl.haar(rng, M, d) * np.logspace(0, -lk, d)[None, :]) @ wl.haar(rng, d, d).T
    Yg = torch.from_numpy(Y).to(DT[dt]).cuda()
    Yh = Yg.double().cpu().numpy()
    handle.set_option("orth_tsqr", 1)
    try:
        Q = handle.orth(Yg).double().cpu().numpy()
    finally:
        handle.set_option("orth_tsqr", 0)
    Qr, _ = oracle.householder_qr(Yh)
    u = 2.0 ** -53 if dt == "f64" else 2.0 ** -24
    assert np.max(np.abs(Q.T @ Q - np.eye(d))) <= 50 * d * u
    assert np.max(np.abs(Q - Qr)) <= 50 * 10.0 ** lk * u * max(1.0, np.sqrt(d))


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_tsqr_decompose_matches_oracle(handle, dt):
    """Option orth_tsqr on full-rank inputs: the whole decomposition with
    Householder orth()s, element-wise against the oracle (dense parity
    tolerances), and flagged RUQLP_FLAG_TSQR."""
    tol = TOLL[dt]
    for m, n, k, p, q in [(1000, 800, 20, 10, 1), (777, 555, 25, 12, 2), (300, 700, 12, 5, 0)]:
        A, _, _, _ = wl.dense_spectral(m + n, m, n, wl.spectrum_gap(min(m, n), k, 1e-2))
        Om = wl.omega(m + 2 * n, n, k + p)
        Ag = torch.from_numpy(A).to(DT[dt]).cuda()
        Aseen = Ag.double().cpu().numpy()
        handle.set_option("orth_tsqr", 1)
        try:
            Q, L, P, flags = handle.decompose(Ag, torch.from_numpy(Om).cuda(), k, p, q)
        finally:
            handle.set_option("orth_tsqr", 0)
        assert flags & ruqlp.FLAG_TSQR
        Q, L, P = (t.double().cpu().numpy() for t in (Q, L, P))
        ref = oracle.ruqlp(Aseen, Om, q)
        l11 = abs(ref["L"][0, 0])
        assert np.max(np.abs(L - ref["L"])) <= tol * l11
        r = oracle.residual_fro_small(Aseen, Q, L, P)
        r0 = oracle.residual_fro_small(Aseen, ref["Q"], ref["L"], ref["P"])
        assert abs(r - r0) <= tol
        assert np.max(np.abs(Q[:, :k] - ref["Q"][:, :k])) <= TOLQ[dt]
        assert np.max(np.abs(P[:, :k] - ref["P"][:, :k])) <= TOLQ[dt]


def test_batch_rank_deficient_items_equal_single(handle):
    """Exactly rank-k items inside an FP32 batch: one that CholeskyQR
    handles and one it flags (d = 280, rerun alone with TSQR); each equals
    ruqlp_decompose on it bitwise, flags included; the full-rank neighbour is
    not flagged."""
    shapes = [(600, 400, 12, 8), (700, 500, 20, 8), (1200, 1000, 260, 20)]
    As = [wl.dense_spectral(40 + i, m, n, wl.spectrum_gap(min(m, n), k, 1e-2))[0]
          for i, (m, n, k, p) in enumerate(shapes)]
    As[1] = _rank_k(41, shapes[1][0], shapes[1][1], shapes[1][2])
    As[2] = _rank_k(42, shapes[2][0], shapes[2][1], shapes[2][2])
    Ag = [torch.from_numpy(A).float().cuda() for A in As]
    Og = [torch.from_numpy(wl.omega(50 + i, n, k + p)).cuda()
          for i, (m, n, k, p) in enumerate(shapes)]
    ks, ps = [s[2] for s in shapes], [s[3] for s in shapes]
    res = handle.decompose_batch(Ag, Og, ks, None, 1, ps=ps)
    for i, (A, om, k, p) in enumerate(zip(Ag, Og, ks, ps)):
        Q, L, P, f = handle.decompose(A, om, k, p, 1, out_dtype=torch.float32)
        assert f == res[i][3], (i, f, res[i][3])
        if i == 0:
            assert f & (ruqlp.FLAG_RANKDEF | ruqlp.FLAG_TSQR) == 0, f
        for x, y in zip(res[i][:3], (Q, L, P)):
            assert torch.equal(x, y), i
