"""The allocation-free brute-force entry point (nhq_brute_force_noalloc).

It serves callers that cannot allocate device memory when they call the
library, so its working memory is a fixed array compiled into the library.
These tests call it through the C ABI and check it against nhq_brute_force on
the same inputs, twice in a row (the fixed array keeps the previous call's
contents), and check that a batch needing more than the fixed array is
refused.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth
from helpers import dev, ids_i64

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nhq():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2203_13601_gb300 import build as B

    B.build()
    import paper_2203_13601_gb300 as m

    m.load_library()
    return m


def _packed(nhq, A):
    out = torch.empty(A.shape[0], dtype=torch.uint32, device="cuda:0")
    nhq.nhq_pack_attributes(dev(A), out)
    return out


@pytest.mark.parametrize("N,nq,k,weights", [(3000, 70, 10, None), (40000, 5, 50, (1.0, 1e4)),
                                            (2500, 33, 7, "filter")])
def test_noalloc_matches_brute_force_twice(nhq, N, nq, k, weights):
    w = synth.int_valued(N, nq, 48, cards=(3, 4, 5), seed=N + nq)
    X, Qv = dev(w.X), dev(w.Qv)
    pa, pq = _packed(nhq, w.A), _packed(nhq, w.QA)
    ref_ids = torch.empty((nq, k), dtype=torch.uint32, device="cuda:0")
    ref_g = torch.empty((nq, k), dtype=torch.float32, device="cuda:0")
    ref_c = torch.empty((nq, k), dtype=torch.uint8, device="cuda:0")
    wts = weights if weights is not None else None
    with nhq.Index.create(X, dev(w.A), weights if isinstance(weights, tuple) else None) as ix:
        nhq.nhq_brute_force(ix.handle, Qv, dev(w.QA), k, ref_ids, ref_g, ref_c,
                            weights="index" if weights is None else wts)
    torch.cuda.synchronize()
    for _ in range(2):  # two calls in a row share the fixed working array
        ids = torch.full((nq, k), 7, dtype=torch.uint32, device="cuda:0")
        g = torch.zeros((nq, k), dtype=torch.float32, device="cuda:0")
        c = torch.zeros((nq, k), dtype=torch.uint8, device="cuda:0")
        nhq.nhq_brute_force_noalloc(X, pa, w.m, Qv, pq, k, ids, g, c, weights=wts)
        torch.cuda.synchronize()
        assert (ids_i64(ids) == ids_i64(ref_ids)).all()
        assert torch.equal(c, ref_c)
        rg, gg = ref_g.cpu().numpy(), g.cpu().numpy()
        fin = np.isfinite(rg)
        assert (np.isfinite(gg) == fin).all()
        assert np.allclose(gg[fin], rg[fin], rtol=1e-5, atol=0)


def test_noalloc_refuses_a_batch_beyond_its_fixed_memory(nhq):
    w = synth.int_valued(40000, 2000, 16, seed=5)
    X, Qv = dev(w.X), dev(w.Qv)
    pa, pq = _packed(nhq, w.A), _packed(nhq, w.QA)
    ids = torch.empty((2000, 256), dtype=torch.uint32, device="cuda:0")
    with pytest.raises(nhq.NHQError) as e:
        nhq.nhq_brute_force_noalloc(X, pa, w.m, Qv, pq, 256, ids)
    assert "scratch bytes" in str(e.value)
    # the same batch in smaller pieces is accepted
    small = torch.empty((100, 256), dtype=torch.uint32, device="cuda:0")
    nhq.nhq_brute_force_noalloc(X, pa, w.m, Qv[:100].contiguous(), pq[:100].contiguous(), 256,
                                small)
    torch.cuda.synchronize()
