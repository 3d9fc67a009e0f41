"""ruqlp_gram_noalloc: the Gram entry point for callers that cannot allocate
device memory (graph capture, host programs that own all device memory,
loops that cannot take cudaMalloc's synchronisation).  It must give the same
G = Y^T Y as ruqlp_gram, the regular entry point, within the tolerance the
Gram tests use (1e-13 ||Y||_F^2), on two calls in a row that share the
library's fixed scratch array.  The file sorts last so that a run stopping at
the first failure has already run every other test."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ruqlp():
    import __graft_entry__ as g
    g.build()
    from paper_2209_12464_gb300 import ruqlp as r
    return r


def _code(r, dt):
    return r.F64 if dt == torch.float64 else r.F32


def test_gram_noalloc_matches_gram_entry_two_calls(ruqlp):
    stream = torch.cuda.current_stream().cuda_stream
    h = ruqlp.Handle(0, stream)
    try:
        rng = np.random.default_rng(2026)
        # calls in a row through the shared scratch: a large one that fills
        # many partial slabs, a smaller one that reuses stale contents, and
        # d = 256 with enough rows that the slab count is clamped to the 8
        # that fill the 4 MiB scratch exactly (8 x 256^2 doubles)
        for M, d, dt in [(20011, 220, torch.float32), (5003, 64, torch.float64),
                         (40000, 256, torch.float32)]:
            Y = torch.from_numpy(rng.standard_normal((M, d))).to(dt).cuda()
            G_ref = h.gram(Y)
            G = torch.full((d, d), float("nan"), dtype=torch.float64, device="cuda")
            st = ruqlp.ruqlp_gram_noalloc(Y.data_ptr(), M, d, Y.stride(0), _code(ruqlp, dt),
                                          G.data_ptr(), stream)
            torch.cuda.synchronize()
            assert st == ruqlp.OK
            tol = 1e-13 * float((Y.double() ** 2).sum())
            assert float((G - G_ref).abs().max()) <= tol
    finally:
        h.close()


def test_gram_noalloc_rejects_sizes_beyond_its_scratch(ruqlp):
    Y = torch.zeros(300, 257, dtype=torch.float32, device="cuda")
    G = torch.empty(257, 257, dtype=torch.float64, device="cuda")
    st = ruqlp.ruqlp_gram_noalloc(Y.data_ptr(), 300, 257, 257, ruqlp.F32, G.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    assert st == ruqlp.ERR_BUDGET
