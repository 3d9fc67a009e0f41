"""GPU tests of the request loop (ruqlp_submit / ruqlp_poll): decompositions
admitted as slots and HBM budget free up, batched when they can be, their
work overlapping on the device.

The property that matters for serving: a request's result is the same alone
and in the mix.  Here it is checked bitwise: small requests against the
batched path on that request alone, wide ones (d = 272, which run alone on
the single-matrix path) against ruqlp_decompose.
"""
import time

import numpy as np
import pytest
import torch

from paper_2209_12464_gb300 import ruqlp
from paper_2209_12464_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as g
    g.build()


def _small_pool(seed, count, dtype=torch.bfloat16):
    shapes = wl.batch_shapes(seed, count=count, m_range=(256, 1500), n_range=(128, 900))
    As, Oms = [], []
    for i, (m, n, k, p) in enumerate(shapes):
        A = wl.dense_lowrank_gauss_torch(seed + i, m, n, k, noise_std=1e-4)
        As.append(wl.aligned_rows(A.to(dtype)))
        Oms.append(wl.omega_torch(seed + 1000 + i, n, k + p))
    torch.cuda.synchronize()  # the request loop's streams do not wait on torch's
    return shapes, As, Oms


def _wait(h, tickets, timeout=120.0):
    t0 = time.time()
    pending = list(tickets)
    while pending:
        pending = [t for t in pending if not h.poll(t)]
        if time.time() - t0 > timeout:
            raise TimeoutError(f"{len(pending)} requests not done")
        time.sleep(0.0005)


def test_serve_mix_equals_alone(built):
    stream = torch.cuda.current_stream().cuda_stream
    server = ruqlp.Handle(0, stream, hbm_budget_bytes=0, max_slots=4)
    alone = ruqlp.Handle(0, stream)
    try:
        shapes, As, Oms = _small_pool(wl.MASTER_SEED + 60, 40)
        big_m, big_n, big_k, big_p = 2048, 1536, 256, 16
        Abig = wl.aligned_rows(wl.dense_lowrank_gauss_torch(7, big_m, big_n, big_k).bfloat16())
        Obig = wl.omega_torch(8, big_n, big_k + big_p)
        torch.cuda.synchronize()
        tickets = []
        for i, ((m, n, k, p), A, om) in enumerate(zip(shapes, As, Oms)):
            tickets.append(("s", i, server.submit(A, om, k, p, 1)))
            if i % 13 == 5:
                tickets.append(("b", i, server.submit(Abig, Obig, big_k, big_p, 2)))
            if i % 7 == 0:
                time.sleep(0.001)  # arrivals while earlier requests run
        _wait(server, [t for _, _, t in tickets])
        for kind, i, t in tickets:
            assert t.flags is not None
            s0, s1, s2 = t.times
            assert 0.0 <= s0 <= s1 <= s2
            if kind == "s":
                m, n, k, p = shapes[i]
                ref = alone.decompose_batch([As[i]], [Oms[i]], [k], p, 1)[0]
            else:
                ref = alone.decompose(Abig, Obig, big_k, big_p, 2, out_dtype=torch.float32)
            for x, y in zip(t.outs, ref[:3]):
                assert torch.equal(x, y), (kind, i)
    finally:
        server.close()
        alone.close()


def test_serve_tight_budget_still_completes(built):
    """A budget that holds about one request at a time: admission waits for
    memory, every request completes and matches its result alone."""
    stream = torch.cuda.current_stream().cuda_stream
    shapes, As, Oms = _small_pool(wl.MASTER_SEED + 61, 12)
    need = max(ruqlp.ruqlp_workspace_bytes(m, n, k + p, ruqlp.BF16) for m, n, k, p in shapes)
    server = ruqlp.Handle(0, stream, hbm_budget_bytes=int(3 * need), max_slots=4)
    alone = ruqlp.Handle(0, stream)
    try:
        tickets = [server.submit(A, om, k, p, 1) for (m, n, k, p), A, om in zip(shapes, As, Oms)]
        _wait(server, tickets)
        for (m, n, k, p), A, om, t in zip(shapes, As, Oms, tickets):
            ref = alone.decompose_batch([A], [om], [k], p, 1)[0]
            for x, y in zip(t.outs, ref[:3]):
                assert torch.equal(x, y)
    finally:
        server.close()
        alone.close()


def test_serve_rejects_oversize_and_invalid(built):
    stream = torch.cuda.current_stream().cuda_stream
    server = ruqlp.Handle(0, stream, hbm_budget_bytes=1 << 20, max_slots=2)
    try:
        A = torch.randn(3000, 2000, device="cuda")
        om = torch.randn(2000, 40, dtype=torch.float64, device="cuda")
        with pytest.raises(ruqlp.RuqlpError) as ei:
            server.submit(A, om, 30, 10, 1)
        assert ei.value.status == ruqlp.ERR_BUDGET
        with pytest.raises(ruqlp.RuqlpError) as ei:
            server.submit(A, om, 0, 40, 1)
        assert ei.value.status == ruqlp.ERR_INVALID
        assert ruqlp.ruqlp_poll(server.h, 12345) == ruqlp.ERR_INVALID
    finally:
        server.close()


def test_serve_fp32_and_mixed_q_groups(built):
    """FP32 and BF16 requests, q = 1 and q = 2, interleaved: each batch holds
    one (dtype, q) group; results equal the batched path alone."""
    stream = torch.cuda.current_stream().cuda_stream
    server = ruqlp.Handle(0, stream, max_slots=3)
    alone = ruqlp.Handle(0, stream)
    try:
        shapes, As, Oms = _small_pool(wl.MASTER_SEED + 62, 16)
        items = []
        for i, ((m, n, k, p), A, om) in enumerate(zip(shapes, As, Oms)):
            Ai = A if i % 2 else wl.aligned_rows(A.float())
            torch.cuda.synchronize()
            q = 1 + (i % 3 == 0)
            items.append((Ai, om, k, p, q, server.submit(Ai, om, k, p, q)))
        _wait(server, [it[-1] for it in items])
        for Ai, om, k, p, q, t in items:
            ref = alone.decompose_batch([Ai], [om], [k], p, q)[0]
            for x, y in zip(t.outs, ref[:3]):
                assert torch.equal(x, y)
    finally:
        server.close()
        alone.close()
