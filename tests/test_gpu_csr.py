"""GPU parity of the CSR path (Section III-D: sparse A, O(sd) per pass).

Products: Y = A X and A^T X with FP32 accumulation against the oracle's FP64
products of the same values (the BF16-valued variant is compared with the
oracle on the rounded values).  Bound per element: 4 sqrt(nnz in the row or
column) u_32 (|A||X|)_ij.  Decompositions: the FP32 tolerances of the dense
path (L and residual within 1e-5 |L_11|, leading-k columns of Q and P within
1e-4).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2209_12464_gb300 import ruqlp
from paper_2209_12464_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def handle():
    import __graft_entry__ as g
    g.build()
    h = ruqlp.Handle(0, torch.cuda.current_stream().cuda_stream)
    yield h
    h.close()


def _dev(A, vdtype):
    return (torch.from_numpy(A["rowptr"]).cuda(), torch.from_numpy(A["colidx"]).cuda(),
            torch.from_numpy(A["values"]).to(vdtype).cuda())


def _seen(A, vals_dev):
    B = dict(A)
    B["values"] = vals_dev.double().cpu().numpy()
    return B


PROD = [  # m, n, density, d
    (3000, 2000, 0.01, 30), (777, 1555, 0.02, 37), (5000, 300, 0.0005, 1), (1200, 900, 0.01, 130),
    (400, 4000, 0.005, 220),
]


@pytest.mark.parametrize("vdtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
@pytest.mark.parametrize("trans", [False, True], ids=["AX", "AtX"])
@pytest.mark.parametrize("case", PROD, ids=[f"{a}x{b}r{c}d{e}" for a, b, c, e in PROD])
def test_csr_product_parity(handle, case, trans, vdtype):
    m, n, dens, d = case
    A = wl.csr_uniform(m + n + d, m, n, dens)
    rp, ci, va = _dev(A, vdtype)
    K = m if trans else n
    X = torch.from_numpy(np.random.default_rng(d).standard_normal((K, d))).float().cuda()
    Y = handle.sketch_csr(rp, ci, va, (m, n), X, trans=trans).double().cpu().numpy()
    As = _seen(A, va)
    Xh = X.double().cpu().numpy()
    ref = oracle.apply_At(As, Xh) if trans else oracle.apply_A(As, Xh)
    absA = dict(As)
    absA["values"] = np.abs(As["values"])
    mag = oracle.apply_At(absA, np.abs(Xh)) if trans else oracle.apply_A(absA, np.abs(Xh))
    kmax = max(1, int(np.max(np.diff(A["rowptr"]))) if not trans else
               int(np.max(np.bincount(A["colidx"], minlength=n))))
    assert np.all(np.abs(Y - ref) <= 4 * math.sqrt(kmax) * U32 * mag + 1e-30)


def test_csr_empty_rows_and_columns(handle):
    """Rows and columns without nonzeros give zero sketch rows."""
    A = wl.csr_uniform(3, 500, 400, 0.002)
    assert np.any(np.diff(A["rowptr"]) == 0)
    rp, ci, va = _dev(A, torch.float32)
    X = torch.randn(400, 16, device="cuda")
    Y = handle.sketch_csr(rp, ci, va, (500, 400), X).cpu().numpy()
    empty = np.diff(A["rowptr"]) == 0
    assert np.all(Y[empty] == 0.0)
    Z = handle.sketch_csr(rp, ci, va, (500, 400), torch.randn(500, 16, device="cuda"),
                          trans=True).cpu().numpy()
    emptyc = np.bincount(A["colidx"], minlength=400) == 0
    assert np.all(Z[emptyc] == 0.0)


DEC = [  # m, n, density, planted rank, scale, k, p, q
    (3000, 2000, 0.02, 10, 10.0, 10, 5, 1), (2500, 3500, 0.01, 6, 20.0, 6, 6, 2),
    (4000, 1500, 0.005, 4, 30.0, 4, 4, 0),
]


@pytest.mark.parametrize("vdtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
@pytest.mark.parametrize("case", DEC, ids=[f"{c[0]}x{c[1]}q{c[7]}" for c in DEC])
def test_csr_decompose_parity(handle, case, vdtype):
    m, n, dens, r, sc, k, p, q = case
    A = wl.csr_uniform(m * 3 + n, m, n, dens, planted_rank=r, planted_scale=sc)
    rp, ci, va = _dev(A, vdtype)
    Om = wl.omega(m + 1, n, k + p)
    Q, L, P, flags = handle.decompose_csr(rp, ci, va, (m, n), torch.from_numpy(Om).cuda(), k, p, q)
    Q, L, P = (t.double().cpu().numpy() for t in (Q, L, P))
    As = _seen(A, va)
    ref = oracle.ruqlp(As, Om, q)
    l11 = abs(ref["L"][0, 0])
    assert np.all(np.triu(L, 1) == 0.0)
    assert np.max(np.abs(L - ref["L"])) <= 1e-5 * l11
    r_gpu = oracle.residual_fro(As, Q, L, P)
    r0 = oracle.residual_fro(As, ref["Q"], ref["L"], ref["P"])
    assert abs(r_gpu - r0) <= 1e-5
    assert np.max(np.abs(Q[:, :k] - ref["Q"][:, :k])) <= 1e-4
    assert np.max(np.abs(P[:, :k] - ref["P"][:, :k])) <= 1e-4


@pytest.mark.parametrize("bad", ["unsorted", "out_of_range", "rowptr", "duplicate"])
def test_csr_invalid_structure_rejected(handle, bad):
    A = wl.csr_uniform(9, 200, 100, 0.05)
    rowptr, colidx = A["rowptr"].copy(), A["colidx"].copy()
    row = int(np.argmax(np.diff(rowptr)))
    a = rowptr[row]
    if bad == "unsorted":
        colidx[a], colidx[a + 1] = colidx[a + 1], colidx[a]
    elif bad == "out_of_range":
        colidx[a] = 100
    elif bad == "rowptr":
        rowptr[5] = rowptr[6] + 1
    elif bad == "duplicate":
        colidx[a + 1] = colidx[a]
    d = 6
    om = torch.randn(100, d, dtype=torch.float64, device="cuda")
    rp = torch.from_numpy(rowptr).cuda()
    ci = torch.from_numpy(colidx).cuda()
    va = torch.from_numpy(A["values"]).float().cuda()
    with pytest.raises(ruqlp.RuqlpError) as ei:
        handle.decompose_csr(rp, ci, va, (200, 100), om, 4, 2, 1)
    assert ei.value.status == ruqlp.ERR_INVALID


def test_csr_full_size_workload_against_oracle(handle):
    """The sparse workload: 200000 x 100000, uniform 0.1 % pattern, N(0,1)
    values plus a planted rank-100 term of scale 10, k=100, p=10, q=1."""
    m, n, k, p, q = 200000, 100000, 100, 10, 1
    A = wl.csr_uniform(wl.MASTER_SEED + 3, m, n, 1e-3, planted_rank=100, planted_scale=10.0)
    rp, ci, va = _dev(A, torch.float32)
    Om = wl.omega(wl.MASTER_SEED + 4, n, k + p)
    Q, L, P, flags = handle.decompose_csr(rp, ci, va, (m, n), torch.from_numpy(Om).cuda(), k, p, q)
    Q, L, P = (t.double().cpu().numpy() for t in (Q, L, P))
    As = _seen(A, va)
    ref = oracle.ruqlp(As, Om, q)
    l11 = abs(ref["L"][0, 0])
    assert np.max(np.abs(L - ref["L"])) <= 1e-5 * l11
    r_gpu = oracle.residual_fro(As, Q, L, P)
    r0 = oracle.residual_fro(As, ref["Q"], ref["L"], ref["P"])
    assert abs(r_gpu - r0) <= 1e-5
    assert np.max(np.abs(Q.T @ Q - np.eye(k + p))) <= 2e-5


def _lowrank_dev(A):
    lr = A["lowrank"]
    return tuple(torch.from_numpy(np.ascontiguousarray(lr[k])).float().cuda() for k in ("X", "D", "Y"))


def _seen_lr(A, vals_dev, lr_dev):
    B = _seen(A, vals_dev)
    B["lowrank"] = {k: t.double().cpu().numpy() for k, t in zip(("X", "D", "Y"), lr_dev)}
    return B


@pytest.mark.parametrize("trans", [False, True], ids=["AX", "AtX"])
def test_csr_lowrank_product_parity(handle, trans):
    """Products with A = S + X D Y^T (CSR plus low-rank term) against the
    oracle's FP64 products of the same FP32 values: the SpMM bound for S plus
    FP32 accumulation over n (or m) terms for the thin products."""
    m, n, r, d = 3000, 2000, 24, 40
    A = wl.csr_lowrank(71, m, n, 0.01, r, 60.0)
    rp, ci, va = _dev(A, torch.float32)
    lr = _lowrank_dev(A)
    K = m if trans else n
    X = torch.from_numpy(np.random.default_rng(3).standard_normal((K, d))).float().cuda()
    Y = handle.sketch_csr(rp, ci, va, (m, n), X, trans=trans, lowrank=lr).double().cpu().numpy()
    As = _seen_lr(A, va, lr)
    Xh = X.double().cpu().numpy()
    ref = oracle.apply_At(As, Xh) if trans else oracle.apply_A(As, Xh)
    assert np.max(np.abs(Y - ref)) <= 64 * math.sqrt(K) * U32 * np.max(np.abs(ref))


@pytest.mark.parametrize("vdtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
def test_csr_lowrank_decompose_parity(handle, vdtype):
    """RU-QLP of a sparse-plus-low-rank input: the FP32 tolerances of the
    sparse path, and the gap after r visible in |diag(L)|."""
    m, n, r, k, p, q = 4000, 2500, 12, 12, 8, 1
    A = wl.csr_lowrank(72, m, n, 0.005, r, 600.0)
    rp, ci, va = _dev(A, vdtype)
    lr = _lowrank_dev(A)
    Om = wl.omega(73, n, k + p)
    Q, L, P, flags = handle.decompose_csr(rp, ci, va, (m, n), torch.from_numpy(Om).cuda(), k, p, q,
                                          lowrank=lr)
    Q, L, P = (t.double().cpu().numpy() for t in (Q, L, P))
    As = _seen_lr(A, va, lr)
    ref = oracle.ruqlp(As, Om, q)
    l11 = abs(ref["L"][0, 0])
    assert np.max(np.abs(L - ref["L"])) <= 1e-5 * l11
    r_gpu = oracle.residual_fro(As, Q, L, P)
    r0 = oracle.residual_fro(As, ref["Q"], ref["L"], ref["P"])
    assert abs(r_gpu - r0) <= 1e-5
    Ld = np.abs(np.diag(L))
    assert np.min(Ld[:r]) > 3.0 * np.max(Ld[r:])
