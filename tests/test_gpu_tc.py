"""GPU parity of the BF16 tensor-core path (tcgen05 products) through the C ABI.

* Product kernel (ruqlp_sketch, Algorithm 1 step 3 / Algorithm 2 / B^T = A^T Q):
  Y = A X or A^T X with A and X rounded to BF16, FP32 accumulation in TMEM,
  against the FP64 product of the same BF16 values (oracle.apply_A /
  apply_At).  Bound per element: 4 sqrt(K) u_32 (|A||X|)_ij, the typical
  size of FP32 accumulation error over K terms (u_32 = 2^-24).
* Whole decomposition (the reduced-precision bar): the relative residual
  ||A - Q L P^T||_F / ||A||_F of the BF16 path is at most 1.05x the FP64
  oracle's on the matrix the GPU was given (A rounded to BF16, widened
  exactly to FP64), at every test size; on the 20000 x 20000 workload also
  against the unrounded FP32 matrix.  The last product B^T = A^T Q takes Q
  as two BF16 parts, so the rounding of Q (2^-9 sqrt(d / m) of ||A||_F,
  which at small m exceeds the oracle's residual) does not enter L.
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


def _bf16(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(torch.bfloat16)


# n a multiple of 8 runs on the tensor cores (16-byte TMA row pitch); the
# 777 x 555 case runs on the CUDA-core BF16 kernel.  Ragged tiles in m, n and
# d, stream-K tails (fewer tiles than SMs, one more tile than a wave) included.
SHAPES = [
    (1000, 800, 30), (777, 552, 37), (777, 555, 37), (300, 7000, 16), (7000, 296, 256),
    (129, 72, 1), (128, 64, 16), (4096, 2048, 72), (19459, 136, 100), (152 * 128 + 5, 96, 224),
]


@pytest.mark.parametrize("trans", [False, True], ids=["AX", "AtX"])
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{a}x{b}d{c}" for a, b, c in SHAPES])
def test_tc_product_parity(handle, shape, trans):
    m, n, d = shape
    rng = np.random.default_rng(m * 7 + n + d)
    A = _bf16(rng.standard_normal((m, n)))
    K = m if trans else n
    X = torch.from_numpy(rng.standard_normal((K, d))).float()
    Y = handle.sketch(A.cuda(), X.cuda(), trans=trans).double().cpu().numpy()
    Ah = A.double().numpy()
    Xh = X.to(torch.bfloat16).double().numpy()
    ref = oracle.apply_At(Ah, Xh) if trans else oracle.apply_A(Ah, Xh)
    mag = (np.abs(Ah).T if trans else np.abs(Ah)) @ np.abs(Xh)
    err = np.abs(Y - ref)
    assert np.all(err <= 4.0 * math.sqrt(K) * U32 * mag + 1e-30), float((err / (mag + 1e-300)).max())


def test_tc_product_matches_cuda_core_kernel_and_is_deterministic(handle):
    m, n, d = 5000, 3000, 64
    rng = np.random.default_rng(3)
    A = _bf16(rng.standard_normal((m, n))).cuda()
    X = torch.from_numpy(rng.standard_normal((n, d))).float().cuda()
    y1 = handle.sketch(A, X)
    y2 = handle.sketch(A, X)
    assert torch.equal(y1, y2)
    handle.set_option("bf16_simt", 1)
    try:
        ys = handle.sketch(A, X)
    finally:
        handle.set_option("bf16_simt", 0)
    mag = (A.double().abs() @ X.to(torch.bfloat16).double().abs())
    assert float(((y1.double() - ys.double()).abs() / mag).max()) <= 8.0 * math.sqrt(n) * U32


def test_tc_product_full_size_sampled(handle):
    """20000 x 20000 BF16 A, d = 220 (the bench's launch configuration): 64
    sampled output rows (A X) and columns (A^T X) against FP64 products."""
    m = n = 20000
    d = 220
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    A = torch.randn(m, n, generator=g, device="cuda").to(torch.bfloat16)
    X = torch.randn(n, d, generator=g, device="cuda")
    rows = np.random.default_rng(1).choice(m, 64, replace=False)
    for trans in (False, True):
        Y = handle.sketch(A, X, trans=trans)
        Ys = Y[rows].double().cpu().numpy()
        Xh = X.to(torch.bfloat16).double().cpu().numpy()
        As = (A[:, rows].T if trans else A[rows]).double().cpu().numpy()
        ref = As @ Xh
        mag = np.abs(As) @ np.abs(Xh)
        assert np.all(np.abs(Ys - ref) <= 4.0 * math.sqrt(n) * U32 * mag)


def _bf16_check(Ag, Om, k, p, q, Q, L, P):
    """The BF16 bar against the FP64 oracle on the same BF16 values: residual
    <= 1.05x the oracle's, orthonormal Q and P, zero upper triangle of L,
    the leading k |L_ii| within 2e-3 |L_11|.  Returns (r, r0)."""
    Aseen = Ag.double().cpu().numpy()
    Q, L, P = (t.double().cpu().numpy() for t in (Q, L, P))
    d = k + p
    assert np.all(np.triu(L, 1) == 0.0)
    assert np.max(np.abs(Q.T @ Q - np.eye(d))) <= 2e-5
    assert np.max(np.abs(P.T @ P - np.eye(d))) <= 2e-5
    ref = oracle.ruqlp(Aseen, Om, q)
    r = oracle.residual_fro(Aseen, Q, L, P)
    r0 = oracle.residual_fro(Aseen, ref["Q"], ref["L"], ref["P"])
    assert r <= 1.05 * r0, (r, r0)
    dl = np.abs(np.abs(np.diag(L))[:k] - np.abs(np.diag(ref["L"]))[:k])
    assert np.max(dl) <= 2e-3 * abs(ref["L"][0, 0])
    return r, r0


def test_bf16_decompose_structure_small(handle):
    m, n, k, p, q = 4000, 3000, 40, 10, 2
    A, _, s, _ = wl.dense_spectral(77, m, n, wl.spectrum_gap(n, k, 1e-2), noise_std=2e-6)
    Om = wl.omega(78, n, k + p)
    Ag = torch.from_numpy(A).to(torch.bfloat16).cuda()
    Q, L, P, flags = handle.decompose(Ag, torch.from_numpy(Om).cuda(), k, p, q)
    _bf16_check(Ag, Om, k, p, q, Q, L, P)


# shapes of the batched workload's range where the rounding of Q in the last
# product used to dominate the residual (small m, large d / m), rows stored
# 16-byte aligned: tensor cores, or the CUDA-core BF16 kernel (bf16_simt)
BAR_SHAPES = [(256, 512, 64, 8, 1), (300, 1000, 48, 8, 1), (256, 136, 64, 8, 2),
              (1024, 600, 30, 8, 0), (700, 333, 40, 8, 1), (4000, 2048, 64, 8, 1)]


@pytest.mark.parametrize("simt", [0, 1], ids=["tc", "cuda_core"])
@pytest.mark.parametrize("shape", BAR_SHAPES, ids=[f"{a}x{b}k{c}p{d}q{e}" for a, b, c, d, e in BAR_SHAPES])
def test_bf16_small_shapes_meet_bar(handle, shape, simt):
    m, n, k, p, q = shape
    A, _, _, _ = wl.dense_spectral(m + 3 * n + k, m, n, wl.spectrum_gap(min(m, n), k, 1e-2))
    Om = wl.omega(m + n, n, k + p)
    Ag = wl.aligned_rows(torch.from_numpy(A).to(torch.bfloat16).cuda())
    handle.set_option("bf16_simt", simt)
    try:
        Q, L, P, flags = handle.decompose(Ag, torch.from_numpy(Om).cuda(), k, p, q)
    finally:
        handle.set_option("bf16_simt", 0)
    _bf16_check(Ag, Om, k, p, q, Q, L, P)


def test_bf16_wide_sketch_column_chunks(handle):
    """d = 272 > 256 (the MMA's widest N): products run as two column chunks,
    orth() as a 9-tile Cholesky; the BF16 bar against the oracle."""
    m, n, k, p, q = 3000, 2400, 256, 16, 1
    A, _, s, _ = wl.dense_spectral(91, m, n, wl.spectrum_gap(n, k, 1e-2), noise_std=2e-6)
    Om = wl.omega(92, n, k + p)
    Ag = torch.from_numpy(A).to(torch.bfloat16).cuda()
    Q, L, P, flags = handle.decompose(Ag, torch.from_numpy(Om).cuda(), k, p, q)
    _bf16_check(Ag, Om, k, p, q, Q, L, P)


def test_tc_wide_product_matches_halves(handle):
    """A 272-column product equals the two products of its column halves
    computed separately (the chunked launch is a column split)."""
    m, n = 1000, 800
    rng = np.random.default_rng(5)
    A = torch.from_numpy(rng.standard_normal((m, n))).to(torch.bfloat16).cuda()
    X = torch.from_numpy(rng.standard_normal((n, 272))).float().cuda()
    Y = handle.sketch(A, X)
    Y1 = handle.sketch(A, X[:, :144].contiguous())
    Y2 = handle.sketch(A, X[:, 144:].contiguous())
    assert torch.equal(Y[:, :144], Y1) and torch.equal(Y[:, 144:], Y2)


def test_bf16_decompose_full_size_residual_vs_fp64_oracle(handle):
    """The bench workload (20000 x 20000, k=200, p=20, q=2, noise std 1e-6):
    BF16 tensor-core residual <= 1.05x the FP64 oracle's on the same A (the
    unrounded FP32 matrix: the BF16 rounding of A itself included)."""
    m = n = 20000
    k, p, q = 200, 20, 2
    sig = wl.spectrum_gap(n, k, 1e-2)
    A32 = wl.dense_spectral_torch(20261, m, n, sig, noise_std=1e-6, device="cuda")
    Om = wl.omega_torch(20262, n, k + p)
    Ab = A32.to(torch.bfloat16)
    Q, L, P, _ = handle.decompose(Ab, Om, k, p, q)
    A64 = A32.double()
    r_gpu = float(torch.linalg.norm(A64 - (Q.double() @ L.double()) @ P.double().T)
                  / torch.linalg.norm(A64))
    Ah = A32.double().cpu().numpy()
    del A64
    ref = oracle.ruqlp(Ah, Om.cpu().numpy(), q)
    r0 = oracle.residual_fro(Ah, ref["Q"], ref["L"], ref["P"])
    assert r_gpu <= 1.05 * r0, (r_gpu, r0)


# column split of the tensor-core products: each 128-row output tile as ns
# items of dp / ns columns (dp / ns a multiple of 16); ragged m and K,
# stream-K tails and the 20000-row workload shape included
SPLIT_SHAPES = [(1000, 800, 32), (19459, 136, 224), (152 * 128 + 5, 96, 128), (300, 7000, 64),
                (4096, 2048, 256), (20000, 2000, 224)]


@pytest.mark.parametrize("ns", [1, 2, 4])
@pytest.mark.parametrize("trans", [False, True], ids=["AX", "AtX"])
@pytest.mark.parametrize("shape", SPLIT_SHAPES, ids=[f"{a}x{b}d{c}" for a, b, c in SPLIT_SHAPES])
def test_tc_product_column_split_parity(handle, shape, trans, ns):
    m, n, d = shape
    if d % (16 * ns):
        pytest.skip("dp / ns must be a multiple of 16")
    rng = np.random.default_rng(m * 3 + n + d + ns)
    A = _bf16(rng.standard_normal((m, n)))
    K = m if trans else n
    X = torch.from_numpy(rng.standard_normal((K, d))).float()
    handle.set_option("tc_nsplit", ns)
    try:
        Y = handle.sketch(A.cuda(), X.cuda(), trans=trans).double().cpu().numpy()
    finally:
        handle.set_option("tc_nsplit", 0)
    Ah = A.double().numpy()
    Xh = X.to(torch.bfloat16).double().numpy()
    ref = oracle.apply_At(Ah, Xh) if trans else oracle.apply_A(Ah, Xh)
    mag = (np.abs(Ah).T if trans else np.abs(Ah)) @ np.abs(Xh)
    err = np.abs(Y - ref)
    assert np.all(err <= 4.0 * math.sqrt(K) * U32 * mag + 1e-30), float((err / (mag + 1e-300)).max())


def test_tuner_file_and_determinism(handle, tmp_path):
    """The product tuner: the first product of a new shape writes its choice
    to the tune file (a valid split and ring depth); a BF16 decomposition of a
    fresh shape is bitwise the same on its first (tuning) and second call;
    reloading the file restores the entries."""
    path = str(tmp_path / "tune.txt")
    assert ruqlp.ruqlp_tune_file(path) == 0
    try:
        m, n, k, p, q = 6000, 4096, 56, 8, 1  # d = 64: splits 1, 2, 4 are all valid
        A, _, _, _ = wl.dense_spectral(123, m, n, wl.spectrum_gap(n, k, 1e-2), noise_std=1e-6)
        Om = torch.from_numpy(wl.omega(124, n, k + p)).cuda()
        Ag = torch.from_numpy(A).to(torch.bfloat16).cuda()
        a = handle.decompose(Ag, Om, k, p, q)
        b = handle.decompose(Ag, Om, k, p, q)
        for x, y in zip(a[:3], b[:3]):
            assert torch.equal(x, y)
        lines = [ln.split() for ln in open(path).read().splitlines() if ln.strip()]
        assert lines, "no tuning entry written"
        shapes = set()
        for ln in lines:
            assert ln[0] == "tc_gemm" and len(ln) == 9
            trans, two, rows, K, dp, ns, stages = (int(v) for v in ln[1:8])
            assert dp == 64 and ns in (1, 2, 4) and (dp // ns) % 16 == 0 and stages >= 2
            shapes.add((trans, two, rows, K))
        # A X (rows m, K n), A^T Y (rows n, K m) and the two-part B^T = A^T Q
        assert {(0, 0, m, n), (1, 0, n, m), (1, 1, n, m)} <= shapes, shapes
        assert ruqlp.ruqlp_tune_file(path) == len(lines)
    finally:
        ruqlp.ruqlp_tune_file(None)
