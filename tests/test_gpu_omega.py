"""Device-generated Omega (a NULL params.omega, Section III-A step 1) against
its host twin: the same counter-based draws, equal up to the last bits of the
FP64 log / cos evaluations (a few ulps), and decompositions that take it
match the ones given the host twin's Omega explicitly."""
import numpy as np
import pytest
import torch

import oracle
from paper_2209_12464_gb300 import ruqlp
from paper_2209_12464_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle():
    import __graft_entry__ as g
    g.build()
    h = ruqlp.Handle(0, torch.cuda.current_stream().cuda_stream)
    yield h
    h.close()


@pytest.mark.parametrize("seed", [0, 20260, (1 << 40) + 12345])
def test_device_omega_matches_host_twin(handle, seed):
    n, d = 3001, 37
    dev = handle.omega(n, d, seed).cpu().numpy()
    host = wl.omega_philox(seed, n, d)
    assert np.max(np.abs(dev - host) / np.maximum(1.0, np.abs(host))) <= 1e-14


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_decompose_with_generated_omega(handle, dtype):
    m, n, k, p, q, seed = 900, 700, 20, 10, 1, 777
    sig = wl.spectrum_gap(min(m, n), k, 1e-2)
    A, _, _, _ = wl.dense_spectral(55, m, n, sig)
    Ag = torch.from_numpy(A).to(dtype).cuda()
    Om = wl.omega_philox(seed, n, k + p)
    a = handle.decompose(Ag, None, k, p, q, seed=seed)
    b = handle.decompose(Ag, torch.from_numpy(Om).cuda(), k, p, q)
    tol = 1e-11 if dtype == torch.float64 else 1e-5
    for x, y in zip(a[:3], b[:3]):
        assert torch.max(torch.abs(x - y)).item() <= tol
    ref = oracle.ruqlp(Ag.double().cpu().numpy(), Om, q)
    L = a[1].double().cpu().numpy()
    assert np.max(np.abs(L - ref["L"])) <= (1e-10 if dtype == torch.float64 else 1e-5)


def test_host_entry_and_batch_with_generated_omega(handle):
    m, n, k, p, q, seed = 500, 400, 12, 6, 1, 31
    A = torch.randn(m, n, dtype=torch.float32)
    d = k + p
    outs = (torch.empty(m, d), torch.empty(d, d), torch.empty(n, d))
    Qh, Lh, Ph, _ = handle.decompose_host(A, None, k, p, q, outs, seed=seed)
    Qd, Ld, Pd, _ = handle.decompose(A.cuda(), None, k, p, q, seed=seed)
    assert torch.equal(Qh, Qd.cpu()) and torch.equal(Lh, Ld.cpu())
    Ab = wl.aligned_rows(A.bfloat16().cuda())
    res = handle.decompose_batch([Ab, Ab], [None, handle.omega(n, d, seed)], [k, k], p, q,
                                 seeds=[seed, 0])
    for x, y in zip(res[0][:3], res[1][:3]):
        assert torch.equal(x, y)
