"""The bounded device waits of the tensor-core kernels, made to run out.

Every mbarrier wait in the tcgen05 kernels is bounded (2 s of %globaltimer);
on expiry the CTA sets the handle's error word, stops issuing work, waits
(bounded) for its own copies and MMAs, frees its tensor memory and returns,
and the call reports RUQLP_ERR_TIMEOUT.  The test hook "test_withhold_stage"
makes the first CTA of a product never load its first ring stage -- a wait
that nothing satisfies -- so that path runs without faulting or hanging the
GPU.  Afterwards the same handle must compute correct products and a correct
decomposition (the timed-out CTA freed its TMEM and left no work behind).
"""
import math
import time

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


def _product_ok(A, X, Y):
    Ah = A.double().cpu().numpy()
    Xh = X.to(torch.bfloat16).double().cpu().numpy()
    ref = oracle.apply_A(Ah, Xh)
    mag = np.abs(Ah) @ np.abs(Xh)
    return np.all(np.abs(Y.double().cpu().numpy() - ref) <= 4.0 * math.sqrt(A.shape[1]) * U32 * mag)


def test_wait_runs_out_then_handle_recovers(handle):
    m, n, d = 4096, 2048, 64
    rng = np.random.default_rng(17)
    A = torch.from_numpy(rng.standard_normal((m, n))).to(torch.bfloat16).cuda()
    X = torch.from_numpy(rng.standard_normal((n, d))).float().cuda()
    handle.set_option("tc_nsplit", 1)
    handle.set_option("test_withhold_stage", 1)
    try:
        t0 = time.time()
        with pytest.raises(ruqlp.RuqlpError) as ei:
            handle.sketch(A, X)
        assert ei.value.status == ruqlp.ERR_TIMEOUT
        assert time.time() - t0 < 60.0
    finally:
        handle.set_option("test_withhold_stage", 0)
        handle.set_option("tc_nsplit", 0)
    # the same handle afterwards: a product and a BF16 decomposition
    assert _product_ok(A, X, handle.sketch(A, X))
    k, p, q = 40, 8, 1
    Aw, _, _, _ = wl.dense_spectral(18, 2000, 1600, wl.spectrum_gap(1600, k, 1e-2), noise_std=1e-6)
    Om = wl.omega(19, 1600, k + p)
    Ag = torch.from_numpy(Aw).to(torch.bfloat16).cuda()
    Q, L, P, flags = handle.decompose(Ag, torch.from_numpy(Om).cuda(), k, p, q)
    Aseen = Ag.double().cpu().numpy()
    ref = oracle.ruqlp(Aseen, Om, q)
    r = oracle.residual_fro(Aseen, Q.double().cpu().numpy(), L.double().cpu().numpy(),
                            P.double().cpu().numpy())
    r0 = oracle.residual_fro(Aseen, ref["Q"], ref["L"], ref["P"])
    assert r <= 1.05 * r0, (r, r0)
