"""The FP64 oracle against what the paper and the mathematics fix (CPU only)."""
import numpy as np
import pytest

import oracle
import pins
from paper_2209_12464_gb300 import workloads as wl


def test_householder_qr_pins():
    assert pins.check_qr(oracle.householder_qr) == []


def test_jacobi_svd_pins():
    assert pins.check_svd(oracle.jacobi_svd) == []


def test_ruqlp_pins():
    assert pins.check_ruqlp(oracle.ruqlp, oracle.ruqlp_paper, oracle.principal_sines,
                            oracle.jacobi_svd) == []


def test_csr_matches_dense():
    assert pins.check_csr(oracle.ruqlp) == []


def test_residual_forms_agree():
    A, _, _, _ = wl.dense_spectral(9, 80, 60, wl.spectrum_gap(60, 5, 0.1))
    out = oracle.ruqlp(A, wl.omega(10, 60, 9), 1)
    a = oracle.residual_fro_small(A, out["Q"], out["L"], out["P"])
    b = oracle.residual_fro(A, out["Q"], out["L"], out["P"])
    assert abs(a - b) <= 1e-9 * a


def test_spectral_norm_power_iteration():
    A, _, s, _ = wl.dense_spectral(2, 40, 30, np.geomspace(5.0, 0.1, 30))
    v = oracle.spectral_norm(lambda x: A @ x, lambda y: A.T @ y, 30, iters=400)
    assert abs(v - 5.0) < 1e-9


def test_principal_sines_closed_form():
    # two planes in R^3 meeting at a known angle
    t = 0.3
    X = np.array([[1.0, 0.0], [0.0, np.cos(t)], [0.0, np.sin(t)]])
    W = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    s = oracle.principal_sines(X, W)
    assert np.allclose(s, [0.0, np.sin(t)], atol=1e-15)
    # tiny angle resolved (cosine form would round to 0)
    e = 1e-11
    X = np.array([[1.0], [e], [0.0]]) / np.sqrt(1 + e * e)
    s = oracle.principal_sines(X, np.array([[1.0], [0.0], [0.0]]))
    assert abs(s[0] - e) < 1e-20


def test_cfg1_oracle_against_generator():
    """1000 x 800 workload (sigma_i = 1 for i <= 20, 1e-3/(i-20) after; k=20,
    p=10, q=1): residual between the Eckart-Young floor and the Theorem 5 bound,
    leading |L_ii| within the Theorem 1 interval."""
    import paper_bounds as pb
    m, n, k, p, q = 1000, 800, 20, 10, 1
    sig = wl.spectrum_gap(800, 20, 1e-3)
    A, U, s, V = wl.dense_spectral(wl.MASTER_SEED + 1, m, n, sig)
    Om = wl.omega(wl.MASTER_SEED + 2, n, k + p)
    out = oracle.ruqlp(A, Om, q)
    rF = np.linalg.norm(A - out["Q"] @ out["L"] @ out["P"].T)
    w = pb.omega_ratio_norm(Om, V[:, :k])
    assert rF >= np.sqrt(np.sum(s[k + p:] ** 2)) * (1 - 1e-9)
    assert rF <= pb.thm5_QQtA(s, k, q, w, "F") * (1 + 1e-9)
    wk = pb.omega_ratio_norm(Om[:, :k], V[:, :k])
    _, s11, _ = oracle.jacobi_svd(out["L"][:k, :k])
    assert np.all(s11 <= s[:k] * (1 + 1e-9))
    cmin = np.sqrt(1 - oracle.principal_sines(out["Q"][:, :k], U[:, :k])[-1] ** 2)
    assert np.all(s11 >= s[:k] * cmin * (1 - 1e-9))
    dl = np.abs(np.diag(out["L"]))
    assert np.max(dl[k:]) <= pb.thm1_upper_22(s, k, q, wk, 2) * (1 + 1e-9)


def test_paper_thm1_lower_bound_counterexample():
    """Theorem 1's lower bound sigma_i(R_11) >= sigma_i / sqrt(1 + delta_i^(4q+4)
    ||Phi2 Phi1^+||^2) fails on this seeded q = 0 case even in its d = k form.
    Its proof bounds the eigenvalues of a compression of a matrix by those of
    a principal submatrix, which interlacing does not give.  The pins use the
    exact inequality sigma_i(L_11) >= sigma_i cos(theta_max(Q_1, U_k)) instead."""
    import paper_bounds as pb
    n, k, p, q = 120, 8, 6, 0
    A, U, s, V = wl.dense_spectral(1000 + n + q + 2 * 31, n, n, wl.spectrum_gap(120, 8, 0.1))
    Om = wl.omega(1000 + n + q + 1 + 2 * 31, n, k + p)
    out = oracle.ruqlp(A, Om, q)
    wk = pb.omega_ratio_norm(Om[:, :k], V[:, :k])
    _, s11, _ = oracle.jacobi_svd(out["L"][:k, :k])
    assert s11[-1] < pb.thm1_lower(s, k, q, wk)[-1] * 0.995
    cmin = np.sqrt(1 - oracle.principal_sines(out["Q"][:, :k], U[:, :k])[-1] ** 2)
    assert np.all(s11 >= s[:k] * cmin * (1 - 1e-9))


@pytest.mark.parametrize("bad", [
    dict(m=5, n=4, d=5), dict(m=5, n=4, d=0), dict(q=-1),
])
def test_oracle_rejects_bad_sizes(bad):
    m, n, d, q = bad.get("m", 6), bad.get("n", 5), bad.get("d", 2), bad.get("q", 0)
    with pytest.raises(ValueError):
        oracle.ruqlp(np.ones((m, n)), np.ones((n, d)), q)


def test_sparse_plus_lowrank_operator_equals_dense_form():
    """A = S + X D Y^T applied as products (Section III-D's cost model kept)
    equals the explicitly formed matrix: products, the whole decomposition and
    the residual."""
    A = wl.csr_lowrank(11, 300, 220, 0.05, 6, 80.0)
    lr = A["lowrank"]
    Dn = wl.csr_to_dense(A) + lr["X"] @ lr["D"] @ lr["Y"].T
    rng = np.random.default_rng(12)
    W = rng.standard_normal((220, 9))
    V = rng.standard_normal((300, 9))
    assert np.max(np.abs(oracle.apply_A(A, W) - Dn @ W)) <= 1e-12 * np.max(np.abs(Dn @ W))
    assert np.max(np.abs(oracle.apply_At(A, V) - Dn.T @ V)) <= 1e-12 * np.max(np.abs(Dn.T @ V))
    Om = wl.omega(13, 220, 10)
    a = oracle.ruqlp(A, Om, 1)
    b = oracle.ruqlp(Dn, Om, 1)
    for key in ("Q", "L", "P"):
        assert np.max(np.abs(a[key] - b[key])) <= 1e-10 * max(1.0, np.max(np.abs(b[key])))
    r1 = oracle.residual_fro(A, a["Q"], a["L"], a["P"])
    r2 = oracle.residual_fro_small(Dn, a["Q"], a["L"], a["P"])
    assert abs(r1 - r2) <= 1e-9
    # the low-rank term dominates: the leading |L_ii| track D (Theorem 1's
    # rank revelation), then drop to the sparse part's level
    s = np.linalg.svd(Dn, compute_uv=False)
    Ld = np.abs(np.diag(a["L"]))
    assert np.all(Ld[:6] >= 0.5 * s[5]) and np.all(Ld[6:] <= 2.0 * s[6])


def test_svd_like_finish_is_an_exact_refactoring():
    """Section III-C, Remark 1: L = U S V^T gives A ~= (Q U) S (P V)^T with the
    same residual; S are L's singular values (LAPACK after sorting), and for
    a gapped spectrum the leading ones approximate A's."""
    A, U0, s0, V0 = wl.dense_spectral(21, 300, 200, wl.spectrum_gap(200, 10, 1e-3))
    Om = wl.omega(22, 200, 16)
    o = oracle.ruqlp(A, Om, 1, finish_paper=2)
    sv = np.linalg.svd(o["L"], compute_uv=False)
    assert np.max(np.abs(o["Sigma"] - sv)) <= 1e-13 * sv[0]
    r1 = oracle.residual_fro_small(A, o["Q"], o["L"], o["P"])
    r2 = oracle.residual_fro_small(A, o["Qsvd"], np.diag(o["Sigma"]), o["Psvd"])
    assert abs(r1 - r2) <= 1e-13
    assert np.max(np.abs(o["Qsvd"].T @ o["Qsvd"] - np.eye(16))) <= 1e-13
    assert np.max(np.abs(o["Sigma"][:10] - s0[:10])) <= 1e-6
    # the leading singular subspaces are the generator's (sigma_1..10 are
    # equal, so only the subspace is determined)
    assert np.max(oracle.principal_sines(o["Qsvd"][:, :10], U0[:, :10])) <= 1e-5
    assert np.max(oracle.principal_sines(o["Psvd"][:, :10], V0[:, :10])) <= 1e-5
