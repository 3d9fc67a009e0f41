"""GPU tests of the batched path (ruqlp_decompose_batch): many independent
RU-QLP decompositions (Section III-A, Algorithms 1-2) of uneven shapes in one
call.

  * parity: every item of an FP32 batch against the FP64 oracle with the FP32
    tolerances of the single-matrix path (L and |diag(L)| within 1e-5 |L_11|,
    residual within 1e-5, leading-k columns of Q and P within 1e-4);
  * batch invariance: every item's Q, L, P are bitwise the single-matrix
    result (FP32; BF16 with CUDA-core products on both sides), eagerly, under
    graph capture and on graph replay;
  * tensor-core batches (BF16 A with 16-byte aligned rows, mixed with
    unaligned items that take the CUDA cores): every item bitwise equal to its
    batch of one, and the BF16 accuracy rule against the oracle (below);
  * the full batched workload (512 matrices, m log-uniform in [256, 4096],
    n in [128, 2048], k in [8, 64], p = 8, q = 1): invariance for all items,
    the oracle on a sample.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2209_12464_gb300 import ruqlp
from paper_2209_12464_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

# (m, n, k, p): single and several 64-column tiles, several 512-row Gram
# slabs, m < n, p = 0, the largest batched d (256), a ragged d (5)
MIX = [(64, 40, 2, 6), (900, 700, 30, 8), (2100, 300, 90, 10), (300, 1200, 20, 8),
       (333, 129, 5, 0), (700, 520, 240, 16), (1500, 1500, 60, 8), (257, 2000, 8, 8),
       (129, 65, 40, 8), (4100, 96, 12, 4)]
Q_ITERS = 1


@pytest.fixture(scope="module")
def handle():
    import __graft_entry__ as g
    g.build()
    h = ruqlp.Handle(0, torch.cuda.current_stream().cuda_stream)
    yield h
    h.close()


def _mix(seed, shapes):
    As, Oms = [], []
    for i, (m, n, k, p) in enumerate(shapes):
        sig = wl.spectrum_gap(min(m, n), k, 1e-2)
        A, _, _, _ = wl.dense_spectral(seed + 17 * i, m, n, sig)
        As.append(A)
        Oms.append(wl.omega(seed + 17 * i + 1, n, k + p))
    return As, Oms


def _pad8(A):
    """A in rows that start on 16-byte boundaries: the layout the
    tensor-core batched product needs."""
    return wl.aligned_rows(A)


def _bf16_bound(r0):
    """The reduced-precision bar: the relative residual is at most 1.05x the
    FP64 oracle's on the same (BF16) values.  The last product B^T = A^T Q
    takes Q as two BF16 parts, so the rounding of Q does not enter L."""
    return 1.05 * r0


def _single(handle, A, om, k, p, q):
    Q, L, P, f = handle.decompose(A, om, k, p, q, out_dtype=torch.float32)
    return Q, L, P


def test_batch_parity_with_oracle(handle):
    As, Oms = _mix(wl.MASTER_SEED + 40, MIX)
    Ag = [torch.from_numpy(A).float().cuda() for A in As]
    Og = [torch.from_numpy(o).cuda() for o in Oms]
    res = handle.decompose_batch(Ag, Og, [s[2] for s in MIX], None, Q_ITERS,
                                 ps=[s[3] for s in MIX])
    for (m, n, k, p), A, om, (Q, L, P, flags) in zip(MIX, Ag, Oms, res):
        Aseen = A.double().cpu().numpy()
        ref = oracle.ruqlp(Aseen, om, Q_ITERS)
        Q, L, P = (t.double().cpu().numpy() for t in (Q, L, P))
        l11 = abs(ref["L"][0, 0])
        d = k + p
        assert flags & ruqlp.FLAG_RANKDEF == 0
        assert np.all(np.triu(L, 1) == 0.0)
        assert np.max(np.abs(L - ref["L"])) <= 1e-5 * l11, (m, n, k, p)
        r = oracle.residual_fro_small(Aseen, Q, L, P)
        r0 = oracle.residual_fro_small(Aseen, ref["Q"], ref["L"], ref["P"])
        assert abs(r - r0) <= 1e-5, (m, n, k, p, r, r0)
        assert np.max(np.abs(Q[:, :k] - ref["Q"][:, :k])) <= 1e-4, (m, n, k, p)
        assert np.max(np.abs(P[:, :k] - ref["P"][:, :k])) <= 1e-4, (m, n, k, p)
        assert np.max(np.abs(Q.T @ Q - np.eye(d))) <= 2e-5
        assert np.max(np.abs(P.T @ P - np.eye(d))) <= 2e-5


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
def test_batch_items_bitwise_equal_single(handle, dtype):
    As, Oms = _mix(wl.MASTER_SEED + 41, MIX)
    Ag = [torch.from_numpy(A).to(dtype).cuda() for A in As]
    Og = [torch.from_numpy(o).cuda() for o in Oms]
    ks, ps = [s[2] for s in MIX], [s[3] for s in MIX]
    runs = []
    handle.set_option("bf16_simt", 1)
    try:
        for _ in range(3):  # eager, captured into a graph, replayed
            runs.append(handle.decompose_batch(Ag, Og, ks, None, Q_ITERS, ps=ps))
        for i, (A, om, k, p) in enumerate(zip(Ag, Og, ks, ps)):
            one = _single(handle, A, om, k, p, Q_ITERS)
            for run in runs:
                for x, y in zip(run[i][:3], one):
                    assert torch.equal(x, y), (i, MIX[i])
    finally:
        handle.set_option("bf16_simt", 0)


def test_batch_graph_off_matches(handle):
    As, Oms = _mix(wl.MASTER_SEED + 42, MIX[:4])
    Ag = [torch.from_numpy(A).float().cuda() for A in As]
    Og = [torch.from_numpy(o).cuda() for o in Oms]
    ks, ps = [s[2] for s in MIX[:4]], [s[3] for s in MIX[:4]]
    a = handle.decompose_batch(Ag, Og, ks, None, 2, ps=ps)
    a2 = handle.decompose_batch(Ag, Og, ks, None, 2, ps=ps)
    handle.set_option("batch_graph", 0)
    try:
        b = handle.decompose_batch(Ag, Og, ks, None, 2, ps=ps)
    finally:
        handle.set_option("batch_graph", 1)
    for x, y, z in zip(a, a2, b):
        for u, v, w in zip(x[:3], y[:3], z[:3]):
            assert torch.equal(u, v) and torch.equal(u, w)


def test_batch_new_inputs_same_shapes_replay(handle):
    """A replayed graph reads the new call's A, Omega and outputs."""
    shapes = MIX[:3]
    ks, ps = [s[2] for s in shapes], [s[3] for s in shapes]
    outs = []
    for seed in (50, 51, 52):
        As, Oms = _mix(wl.MASTER_SEED + seed, shapes)
        Ag = [torch.from_numpy(A).float().cuda() for A in As]
        Og = [torch.from_numpy(o).cuda() for o in Oms]
        outs.append((Ag, Og, handle.decompose_batch(Ag, Og, ks, None, 1, ps=ps)))
    for Ag, Og, res in outs:
        for A, om, k, p, r in zip(Ag, Og, ks, ps, res):
            one = _single(handle, A, om, k, p, 1)
            for x, y in zip(r[:3], one):
                assert torch.equal(x, y)


def test_batch_tensor_core_items(handle):
    """BF16 batch, half the items in 16-byte aligned storage (tensor cores),
    the rest unaligned (CUDA cores): each item bitwise equals its batch of
    one, on eager, captured and replayed calls; accuracy against the oracle
    by the BF16 rule."""
    As, Oms = _mix(wl.MASTER_SEED + 43, MIX)
    Ag = []
    for i, A in enumerate(As):
        t = torch.from_numpy(A).bfloat16().cuda()
        Ag.append(_pad8(t) if i % 2 == 0 else t)
    Og = [torch.from_numpy(o).cuda() for o in Oms]
    ks, ps = [s[2] for s in MIX], [s[3] for s in MIX]
    runs = [handle.decompose_batch(Ag, Og, ks, None, Q_ITERS, ps=ps) for _ in range(3)]
    for i in range(len(MIX)):
        one = handle.decompose_batch([Ag[i]], [Og[i]], [ks[i]], ps[i], Q_ITERS)[0]
        for run in runs:
            for x, y in zip(run[i][:3], one[:3]):
                assert torch.equal(x, y), (i, MIX[i])
    for i, ((m, n, k, p), om) in enumerate(zip(MIX, Oms)):
        Q, L, P = (t.double().cpu().numpy() for t in runs[0][i][:3])
        A64 = Ag[i].double().cpu().numpy()  # the BF16 values the GPU saw
        ref = oracle.ruqlp(A64, om, Q_ITERS)
        r = oracle.residual_fro_small(A64, Q, L, P)
        r0 = oracle.residual_fro_small(A64, ref["Q"], ref["L"], ref["P"])
        assert r <= _bf16_bound(r0), (i, MIX[i], r, r0)
        l11 = abs(ref["L"][0, 0])
        assert np.max(np.abs(np.abs(np.diag(L))[:k] - np.abs(np.diag(ref["L"]))[:k])) <= 2e-2 * l11
        d = k + p
        assert np.max(np.abs(Q.T @ Q - np.eye(d))) <= 2e-5
        assert np.max(np.abs(P.T @ P - np.eye(d))) <= 2e-5


# BF16 items for the tensor-core CholeskyQR passes (dp <= 80): one and two
# 32-row chunks, several 512-row Gram slabs and 1024-row units, d = 80 (the
# widest such item) beside d = 81 (CUDA-core passes in the same batch), a
# partial 128-row sub-tile, and a 4-row last unit
TCO = [(40, 300, 10, 6), (3000, 200, 60, 12), (1500, 2500, 70, 10), (700, 900, 73, 8),
       (5000, 120, 20, 8), (129, 4100, 30, 8), (33, 64, 8, 8)]


def test_batch_tc_orth_items(handle):
    """BF16 batch whose CholeskyQR passes run on the tensor cores (option
    batch_orth_tc: the six-part BF16 split of Y^T Y and Q = Y R^{-1},
    Section II-A): every item bitwise equals its batch of one; accuracy
    against the oracle by the BF16 rule; |diag(L)| within 1e-4 |L_11| of the
    same batch with the default CUDA-core passes."""
    As, Oms = _mix(wl.MASTER_SEED + 44, TCO)
    Ag = [_pad8(torch.from_numpy(A).bfloat16().cuda()) for A in As]
    Og = [torch.from_numpy(o).cuda() for o in Oms]
    ks, ps = [s[2] for s in TCO], [s[3] for s in TCO]
    cc = handle.decompose_batch(Ag, Og, ks, None, Q_ITERS, ps=ps)
    handle.set_option("batch_orth_tc", 1)
    try:
        res = handle.decompose_batch(Ag, Og, ks, None, Q_ITERS, ps=ps)
        for i in range(len(TCO)):
            one = handle.decompose_batch([Ag[i]], [Og[i]], [ks[i]], ps[i], Q_ITERS)[0]
            for x, y in zip(res[i][:3], one[:3]):
                assert torch.equal(x, y), (i, TCO[i])
    finally:
        handle.set_option("batch_orth_tc", 0)
    for i, ((m, n, k, p), om) in enumerate(zip(TCO, Oms)):
        assert res[i][3] & ruqlp.FLAG_RANKDEF == 0
        Q, L, P = (t.double().cpu().numpy() for t in res[i][:3])
        Lc = cc[i][1].double().cpu().numpy()
        A64 = Ag[i].double().cpu().numpy()
        ref = oracle.ruqlp(A64, om, Q_ITERS)
        r = oracle.residual_fro_small(A64, Q, L, P)
        r0 = oracle.residual_fro_small(A64, ref["Q"], ref["L"], ref["P"])
        assert r <= _bf16_bound(r0), (i, TCO[i], r, r0)
        l11 = abs(ref["L"][0, 0])
        assert np.max(np.abs(np.abs(np.diag(L))[:k] - np.abs(np.diag(ref["L"]))[:k])) <= 2e-2 * l11
        assert np.max(np.abs(np.abs(np.diag(L))[:k] - np.abs(np.diag(Lc))[:k])) <= 1e-4 * l11, i
        d = k + p
        assert np.max(np.abs(Q.T @ Q - np.eye(d))) <= 2e-5, i
        assert np.max(np.abs(P.T @ P - np.eye(d))) <= 2e-5, i


@pytest.mark.parametrize("bad", ["mixed_dtype", "mixed_q", "d289", "empty", "f64"])
def test_batch_invalid_rejected(handle, bad):
    A1 = torch.randn(300, 280, device="cuda")
    A2 = torch.randn(200, 150, device="cuda")
    o1 = torch.randn(280, 10, dtype=torch.float64, device="cuda")
    o2 = torch.randn(150, 10, dtype=torch.float64, device="cuda")
    As, Os, ks, qs = [A1, A2], [o1, o2], [6, 6], None
    if bad == "mixed_dtype":
        As[1] = A2.bfloat16()
    elif bad == "f64":
        As = [A1.double(), A2.double()]
    elif bad == "d289":
        As[0] = torch.randn(600, 560, device="cuda")
        Os[0] = torch.randn(560, 293, dtype=torch.float64, device="cuda")
        ks[0] = 289
    elif bad == "mixed_q":
        qs = [1, 2]
    if bad == "empty":
        st = ruqlp.ruqlp_decompose_batch(handle.h, 0, None, None, None)
        assert st == ruqlp.ERR_INVALID
        return
    with pytest.raises(ruqlp.RuqlpError) as ei:
        handle.decompose_batch(As, Os, ks, 4, 1, qs=qs)
    assert ei.value.status == ruqlp.ERR_INVALID


@pytest.mark.slow
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16], ids=["f32", "bf16"])
def test_batched_workload_512(handle, dtype):
    """The batched workload (rows in 16-byte aligned storage, as the bench
    lays them out).  FP32: all 512 items bitwise equal ruqlp_decompose.
    BF16: tensor-core batch; 16 sampled items bitwise equal their batch of
    one; then the CUDA-core BF16 batch bitwise equals ruqlp_decompose for all
    512.  Six sampled items against the oracle (FP32 tolerances; BF16 rule)."""
    shapes = wl.batch_shapes(wl.MASTER_SEED + 4)
    A32 = [wl.dense_spectral_torch(wl.MASTER_SEED + 400 + i, m, n,
                                   wl.spectrum_gap(min(m, n), k, 1e-2))
           for i, (m, n, k, p) in enumerate(shapes)]
    Ag = [_pad8(a.to(dtype)) for a in A32]
    Og = [wl.omega_torch(wl.MASTER_SEED + 1400 + i, n, k + p)
          for i, (m, n, k, p) in enumerate(shapes)]
    ks, ps = [s[2] for s in shapes], [s[3] for s in shapes]
    res = handle.decompose_batch(Ag, Og, ks, None, 1, ps=ps)
    rng = np.random.default_rng(7)
    if dtype == torch.bfloat16:
        for i in rng.choice(len(shapes), 16, replace=False):
            one = handle.decompose_batch([Ag[i]], [Og[i]], [ks[i]], ps[i], 1)[0]
            for x, y in zip(res[i][:3], one[:3]):
                assert torch.equal(x, y), (i, shapes[i])
    handle.set_option("bf16_simt", 1)
    try:
        simt = res if dtype == torch.float32 else handle.decompose_batch(Ag, Og, ks, None, 1,
                                                                           ps=ps)
        for i in range(len(shapes)):
            one = _single(handle, Ag[i], Og[i], ks[i], ps[i], 1)
            for x, y in zip(simt[i][:3], one):
                assert torch.equal(x, y), (i, shapes[i])
    finally:
        handle.set_option("bf16_simt", 0)
    for i in rng.choice(len(shapes), 6, replace=False):
        m, n, k, p = shapes[i]
        om = Og[i].cpu().numpy()
        Q, L, P = (t.double().cpu().numpy() for t in res[i][:3])
        if dtype == torch.float32:
            Aseen = Ag[i].double().cpu().numpy()
            ref = oracle.ruqlp(Aseen, om, 1)
            l11 = abs(ref["L"][0, 0])
            assert np.max(np.abs(L - ref["L"])) <= 1e-5 * l11
            r = oracle.residual_fro_small(Aseen, Q, L, P)
            r0 = oracle.residual_fro_small(Aseen, ref["Q"], ref["L"], ref["P"])
            assert abs(r - r0) <= 1e-5
        else:
            A64 = Ag[i].double().cpu().numpy()  # the BF16 values the GPU saw
            ref = oracle.ruqlp(A64, om, 1)
            r = oracle.residual_fro_small(A64, Q, L, P)
            r0 = oracle.residual_fro_small(A64, ref["Q"], ref["L"], ref["P"])
            assert r <= _bf16_bound(r0), (i, shapes[i], r, r0)
