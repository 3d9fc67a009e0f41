"""GPU parity of the dense RU-QLP path against the FP64 oracle, through the C ABI.

Tolerances (stated per result, Section III-A outputs):
  * FP64 path: L element-wise and |diag(L)| within 1e-10 |L_11|; relative
    residual ||A - Q L P^T||_F / ||A||_F within 1e-10 of the oracle's.
  * FP32 path: the same at 1e-5.
  * Q and P: the leading k columns element-wise within 1e-9 (FP64) / 1e-4
    (FP32); they span the well-separated dominant subspaces, so they are
    determined to about u * sigma_1 / (sigma_k - sigma_{k+1}).  The trailing
    p columns are checked through the residual and orthonormality instead
    (their sensitivity grows with kappa of the sketch).
The oracle runs on the exact values the GPU sees (A rounded to the compute
dtype, then widened to float64).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_12464_gb300 import ruqlp
from paper_2209_12464_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-10, torch.float32: 1e-5}
TOLQ = {torch.float64: 1e-9, torch.float32: 1e-4}
TOLO = {torch.float64: 1e-12, torch.float32: 2e-5}

CASES = [
    # name, m, n, k, p, q, spectrum tail
    ("cfg1-1000x800", 1000, 800, 20, 10, 1, 1e-3),
    ("ragged-777x555-q2", 777, 555, 25, 12, 2, 1e-2),
    ("wide-300x700", 300, 700, 12, 5, 1, 1e-2),
    ("q0-640x512", 640, 512, 16, 8, 0, 1e-2),
    ("k1-p0-200x150", 200, 150, 1, 0, 1, 1e-2),
    ("p0-500x400-q2", 500, 400, 30, 0, 2, 1e-2),
    ("tall-3000x200-d64", 3000, 200, 48, 16, 1, 1e-2),
    ("d280-1500x1200", 1500, 1200, 256, 24, 1, 1e-2),
    ("tall-9000x700-tcgram", 9000, 700, 100, 20, 1, 1e-2),
    # the widest sketch the ABI accepts (d = 512) and a ragged d past the
    # 288-column blocked Cholesky (one-CTA Cholesky and row solve there)
    ("d512-1500x1200", 1500, 1200, 480, 32, 1, 1e-2),
    ("d417-1300x900", 1300, 900, 400, 17, 1, 1e-2),
]


@pytest.fixture(scope="module")
def handle():
    import __graft_entry__ as g
    g.build()
    h = ruqlp.Handle(0, torch.cuda.current_stream().cuda_stream)
    yield h
    h.close()


def _case(name, m, n, k, p, q, tail, seed):
    sig = wl.spectrum_gap(min(m, n), k, tail)
    A, _, _, _ = wl.dense_spectral(seed, m, n, sig)
    Om = wl.omega(seed + 1, n, k + p)
    return A, Om


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_dense_parity(handle, case, dtype):
    name, m, n, k, p, q, tail = case
    A, Om = _case(*case, seed=wl.MASTER_SEED + 11 * m + n)
    Ag = torch.from_numpy(A).to(dtype).cuda()
    Aseen = Ag.double().cpu().numpy()
    ref = oracle.ruqlp(Aseen, Om, q)
    Q, L, P, flags = handle.decompose(Ag, torch.from_numpy(Om).cuda(), k, p, q)
    torch.cuda.synchronize()
    Q, L, P = (t.double().cpu().numpy() for t in (Q, L, P))
    tol = TOL[dtype]
    l11 = abs(ref["L"][0, 0])
    d = k + p
    assert flags & ruqlp.FLAG_RANKDEF == 0
    assert np.all(np.triu(L, 1) == 0.0)
    assert np.max(np.abs(L - ref["L"])) <= tol * l11, np.max(np.abs(L - ref["L"])) / l11
    assert np.max(np.abs(np.abs(np.diag(L)) - np.abs(np.diag(ref["L"])))) <= tol * l11
    r = oracle.residual_fro_small(Aseen, Q, L, P)
    r0 = oracle.residual_fro_small(Aseen, ref["Q"], ref["L"], ref["P"])
    assert abs(r - r0) <= tol, (r, r0)
    assert np.max(np.abs(Q[:, :k] - ref["Q"][:, :k])) <= TOLQ[dtype]
    assert np.max(np.abs(P[:, :k] - ref["P"][:, :k])) <= TOLQ[dtype]
    assert np.max(np.abs(Q.T @ Q - np.eye(d))) <= TOLO[dtype]
    assert np.max(np.abs(P.T @ P - np.eye(d))) <= TOLO[dtype]


def test_host_entry_matches_device_entry(handle):
    m, n, k, p, q = 900, 700, 15, 7, 1
    A, Om = _case("host", m, n, k, p, q, 1e-2, seed=4242)
    d = k + p
    Ah = torch.from_numpy(A).pin_memory()
    Omh = torch.from_numpy(Om).pin_memory()
    outs = (torch.empty(m, d, dtype=torch.float64).pin_memory(),
            torch.empty(d, d, dtype=torch.float64).pin_memory(),
            torch.empty(n, d, dtype=torch.float64).pin_memory())
    Qh, Lh, Ph, _ = handle.decompose_host(Ah, Omh, k, p, q, outs)
    Qd, Ld, Pd, _ = handle.decompose(Ah.cuda(), Omh.cuda(), k, p, q)
    torch.cuda.synchronize()
    assert torch.equal(Qh, Qd.cpu()) and torch.equal(Lh, Ld.cpu()) and torch.equal(Ph, Pd.cpu())


def test_repeat_is_bitwise_deterministic(handle):
    A, Om = _case("det", 1500, 1100, 30, 10, 2, 1e-2, seed=99)
    Ag = torch.from_numpy(A).float().cuda()
    Omg = torch.from_numpy(Om).cuda()
    a = handle.decompose(Ag, Omg, 30, 10, 2)
    b = handle.decompose(Ag, Omg, 30, 10, 2)
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)


@pytest.mark.parametrize("bad", ["k0", "pneg", "qneg", "dbig", "nullout", "d513"])
def test_invalid_arguments_rejected(handle, bad):
    m, n = 64, 48
    A = torch.randn(m, n, dtype=torch.float64, device="cuda")
    k, p, q = 4, 2, 1
    om = torch.randn(n, k + p, dtype=torch.float64, device="cuda")
    if bad == "k0":
        k = 0
    elif bad == "pneg":
        p = -1
    elif bad == "qneg":
        q = -1
    elif bad == "dbig":
        k, p = 40, 10
    elif bad == "d513":
        A = torch.randn(600, 600, dtype=torch.float64, device="cuda")
        k, p = 500, 13
    d = max(k + p, 1)
    Q = torch.empty(A.shape[0], d, dtype=torch.float64, device="cuda")
    L = torch.empty(d, d, dtype=torch.float64, device="cuda")
    P = torch.empty(A.shape[1], d, dtype=torch.float64, device="cuda")
    M = ruqlp.Matrix(0, ruqlp.Dense(A.shape[0], A.shape[1], A.shape[1], ruqlp.F64,
                                    A.data_ptr()), ruqlp.Csr())
    prm = ruqlp.Params(k, p, q, ruqlp.F64, om.data_ptr(), 0)
    out = ruqlp.Outputs(0 if bad == "nullout" else Q.data_ptr(), L.data_ptr(), P.data_ptr(),
                        ruqlp.F64, 0)
    st = ruqlp.ruqlp_decompose(handle.h, M, prm, out)
    assert st == ruqlp.ERR_INVALID
    assert ruqlp.ruqlp_last_error(handle.h) != ""


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("shape", [(1000, 30), (20011, 220), (77, 77), (5, 1), (3000, 300)])
def test_gram_entry_matches_fp64_products(handle, shape, dtype):
    """ruqlp_gram: G = Y^T Y with exact FP64 products; compared with numpy's
    FP64 product of the same (rounded) values, relative to ||Y||_F^2."""
    M, d = shape
    Y = torch.from_numpy(np.random.default_rng(M + d).standard_normal((M, d))).to(dtype).cuda()
    G = handle.gram(Y).cpu().numpy()
    Yh = Y.double().cpu().numpy()
    ref = Yh.T @ Yh
    assert np.max(np.abs(G - ref)) <= 1e-13 * np.sum(Yh * Yh)
    assert np.array_equal(G, G.T)


ORTH_CASES = [  # M, d, log10 kappa
    (1000, 30, 1), (1000, 30, 5), (20011, 220, 3), (5003, 64, 6), (300, 300, 2), (129, 1, 0),
    (777, 37, 4), (4096, 272, 3), (9000, 100, 5), (16384, 256, 2), (8192, 17, 3),
    # tall FP32 Y on the tensor cores: 152 equal row ranges of 256 rows (two
    # full sub-tiles), of 257 (three sub-tiles, the last one row) and of 395
    (38912, 64, 2), (38913, 64, 2), (60013, 96, 3),
    # d past the blocked Cholesky's 288 columns, up to the ABI's 512
    (2000, 512, 3), (3001, 417, 2), (12000, 300, 3),
    # orthonormal Y: every pass sees a Gram near I, and the last one takes
    # the first-order factor (several diagonal tiles; tall: tensor cores)
    (4096, 96, 0), (20011, 220, 0), (1000, 288, 0),
]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("case", ORTH_CASES, ids=[f"{a}x{b}k1e{c}" for a, b, c in ORTH_CASES])
def test_orth_matches_householder_q(handle, case, dtype):
    """ruqlp_orth (CholeskyQR2 / shifted CholeskyQR3) against the oracle's
    Householder Q of the same (rounded) Y.  Q is unique for full column rank
    (diag R > 0); column j is determined to about kappa_j u, so the bound is
    50 kappa u with kappa = sigma_1 / sigma_d of Y."""
    M, d, lk = case
    rng = np.random.default_rng(M + d + lk)
    Uy = wl.haar(rng, M, d)
    Vy = wl.haar(rng, d, d)
    Y = (Uy * np.logspace(0, -lk, d)[None, :]) @ Vy.T
    Yg = torch.from_numpy(Y).to(dtype).cuda()
    Yh = Yg.double().cpu().numpy()
    Q = handle.orth(Yg).double().cpu().numpy()
    Qr, Rr = oracle.householder_qr(Yh)
    u = 2.0 ** -53 if dtype == torch.float64 else 2.0 ** -24
    kappa = 10.0 ** lk
    assert np.max(np.abs(Q.T @ Q - np.eye(d))) <= 50 * d * u
    assert np.max(np.abs(Q - Qr)) <= 50 * kappa * u * max(1.0, np.sqrt(d))


@pytest.mark.parametrize("case", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_light_and_full_intermediate_orth_agree(handle, case):
    """Intermediate orth() results with two CholeskyQR passes (default) and
    with the three passes of a final basis (option orth_full) give the same
    Q, L, P within the FP32 tolerance (exact arithmetic: identical, the
    bases differ by upper-triangular factors)."""
    name, m, n, k, p, q, tail = case
    A, Om = _case(*case, seed=wl.MASTER_SEED + 11 * m + n)
    Ag = torch.from_numpy(A).float().cuda()
    Og = torch.from_numpy(Om).cuda()
    a = [t.double().cpu().numpy() for t in handle.decompose(Ag, Og, k, p, q)[:3]]
    handle.set_option("orth_full", 1)
    try:
        b = [t.double().cpu().numpy() for t in handle.decompose(Ag, Og, k, p, q)[:3]]
    finally:
        handle.set_option("orth_full", 0)
    l11 = abs(b[1][0, 0])
    assert np.max(np.abs(a[1] - b[1])) <= 1e-5 * l11
    assert np.max(np.abs(a[0][:, :k] - b[0][:, :k])) <= 1e-4


@pytest.mark.parametrize("shape", [(9000, 700, 100, 20, 1), (12288, 8500, 120, 16, 2),
                                   (8192, 8192, 230, 26, 1)],
                         ids=["Ytall", "YZtall-q2", "d256"])
def test_tensor_core_orth_matches_cuda_core_orth(handle, shape):
    """orth() of tall Y and Z on the tensor cores (three-way BF16 split Gram
    and Q = Y R^{-1}) against the CUDA-core FP32 Gram and blocked triangular
    solve (option orth_simt).  Compared where the
    results are well determined whatever the rounding: the singular values of L (those of Q^T A P depend
    on the spans of Q and P only), the leading-k subspaces of Q and P (largest
    principal-angle sine), orthonormality, and the relative residual.  Single
    columns of Q and entries of L are basis-dependent: Y after the power step
    has kappa ~ 1e3, so they move by ~ kappa u between any two FP32
    orthogonalisations."""
    m, n, k, p, q = shape
    A = wl.dense_lowrank_gauss_torch(wl.MASTER_SEED + m + n, m, n, k, noise_std=1e-4)
    Ag = wl.aligned_rows(A.bfloat16())
    Og = wl.omega_torch(wl.MASTER_SEED + 5 * m, n, k + p)
    a = handle.decompose(Ag, Og, k, p, q)[:3]
    handle.set_option("orth_simt", 1)
    try:
        b = handle.decompose(Ag, Og, k, p, q)[:3]
    finally:
        handle.set_option("orth_simt", 0)
    d = k + p
    A64 = Ag.double()
    res = []
    for Q, L, P in (a, b):
        R = A64 - Q.double() @ L.double() @ P.double().T
        res.append(float(torch.linalg.norm(R) / torch.linalg.norm(A64)))
    a = [t.double().cpu().numpy() for t in a]
    b = [t.double().cpu().numpy() for t in b]
    sa, sb = np.linalg.svd(a[1], compute_uv=False), np.linalg.svd(b[1], compute_uv=False)
    ds = np.max(np.abs(sa - sb)) / sb[0]
    assert ds <= 1e-5, ds
    for x, y in ((a[0], b[0]), (a[2], b[2])):
        U, V = x[:, :k], y[:, :k]
        sin = np.linalg.norm(V - U @ (U.T @ V), 2)
        assert sin <= 1e-4, sin
        assert np.max(np.abs(x.T @ x - np.eye(d))) <= 50 * d * 2.0 ** -24
    assert abs(res[0] - res[1]) <= 1e-5 * max(res[1], 1e-3), res


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("case", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_finish_paper_matches_oracle(handle, case, dtype):
    """finish_paper: Q P~ and R~ of [P~, R~] = qr(L) (Algorithm 1 step 5);
    diag(R~) are the paper's L-values of A^T.  Same tolerances as the dense
    parity test; A ~= (Q P~) R~ P^T."""
    name, m, n, k, p, q, tail = case
    A, Om = _case(*case, seed=wl.MASTER_SEED + 11 * m + n)
    Ag = torch.from_numpy(A).to(dtype).cuda()
    Aseen = Ag.double().cpu().numpy()
    ref = oracle.ruqlp(Aseen, Om, q, finish_paper=True)
    Qh, R, P, _ = handle.decompose(Ag, torch.from_numpy(Om).cuda(), k, p, q, finish_paper=True)
    Qh, R, P = (t.double().cpu().numpy() for t in (Qh, R, P))
    tol = TOL[dtype]
    r11 = abs(ref["Rtilde"][0, 0])
    assert np.all(np.tril(R, -1) == 0.0)
    assert np.max(np.abs(R - ref["Rtilde"])) <= tol * r11
    r = oracle.residual_fro_small(Aseen, Qh, R, P)
    r0 = oracle.residual_fro_small(Aseen, ref["Qhat"], ref["Rtilde"], ref["P"])
    assert abs(r - r0) <= tol
    assert np.max(np.abs(Qh[:, :k] - ref["Qhat"][:, :k])) <= TOLQ[dtype] * 10


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[6]], ids=[CASES[0][0], CASES[1][0],
                                                                     CASES[6][0]])
def test_svd_finish_matches_oracle(handle, case, dtype):
    """finish_paper = 2 (Section III-C, Remark 1): L = diag(S) descending,
    S against the oracle's Jacobi SVD of its L (FP64: 1e-10 |L_11|, FP32:
    1e-5), Q and P orthonormal, residual equal to the oracle's; singular
    vectors of well-separated values match up to sign."""
    name, m, n, k, p, q, tail = case
    A, Om = _case(*case, seed=wl.MASTER_SEED + 7 * m + n)
    Ag = torch.from_numpy(A).to(dtype).cuda()
    Aseen = Ag.double().cpu().numpy()
    ref = oracle.ruqlp(Aseen, Om, q, finish_paper=2)
    Q, L, P, flags = handle.decompose(Ag, torch.from_numpy(Om).cuda(), k, p, q, finish_paper=2)
    Q, L, P = (t.double().cpu().numpy() for t in (Q, L, P))
    d = k + p
    tol = TOL[dtype]
    S = np.diag(L)
    assert np.all(L - np.diag(S) == 0.0)
    assert np.all(np.diff(S) <= 0.0)
    assert np.max(np.abs(S - ref["Sigma"])) <= tol * ref["Sigma"][0]
    assert np.max(np.abs(Q.T @ Q - np.eye(d))) <= TOLO[dtype] * 10
    assert np.max(np.abs(P.T @ P - np.eye(d))) <= TOLO[dtype] * 10
    r = oracle.residual_fro_small(Aseen, Q, L, P)
    r0 = oracle.residual_fro_small(Aseen, ref["Qsvd"], np.diag(ref["Sigma"]), ref["Psvd"])
    assert abs(r - r0) <= tol
    # tail singular values are distinct: their vectors are determined up to sign
    sv = ref["Sigma"]
    for j in range(k, d - 1):
        if min(sv[j - 1] - sv[j], sv[j] - sv[j + 1]) > 1e-3 * sv[j]:
            c = abs(np.dot(Q[:, j], ref["Qsvd"][:, j]))
            assert c >= 1.0 - (1e-6 if dtype == torch.float64 else 1e-2), (j, c)
