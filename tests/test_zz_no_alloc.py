"""The allocation-free brute-force entry point (nhq_brute_force_noalloc).

It serves callers that cannot allocate device memory when they call the
library (their device memory belongs to another allocator or a pool reserved
at start-up, or their hot path must not touch an allocator), so its working
memory is a fixed array compiled into the library.  These tests call it
through the C ABI and check it against the oracle's exact top-k (Def. 2 with
Eq. 6; for the filter weighting the hybrid ground truth of Sec. 6.1) and against
nhq_brute_force on the same inputs, twice in a row (the fixed array keeps the
previous call's contents), check
that the second call changes the device's free memory by nothing, and check
that a batch needing more than the fixed array is refused without writing
anything.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import dev, ids_i64

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIXED_BYTES = 16 << 20  # the library's fixed working array
TQ, TN = 32, 128        # queries per CTA and objects per tile of the brute-force kernel


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


def _split_bytes(N, Q, k, sms):
    """Bytes of per-slice lists the split path needs: the batch is split over the objects
    into S slices so that about two CTAs run per SM, with at least 8 tiles per slice."""
    tiles = -(-Q // TQ)
    S = max(1, min(-(-2 * sms // tiles), -(-N // (8 * TN)), 32))
    return 0 if S == 1 else Q * S * k * 8


def test_noalloc_first_call_with_no_queries_does_the_set_up(nhq):
    # a call with Q = 0 only looks up the fixed array on this device (the start-up call)
    e = torch.empty(0, dtype=torch.float32, device="cuda:0")
    x = torch.zeros((8, 4), dtype=torch.float32, device="cuda:0")
    pa = torch.zeros(8, dtype=torch.uint32, device="cuda:0")
    ids = torch.empty((0, 1), dtype=torch.uint32, device="cuda:0")
    nhq.nhq_brute_force_noalloc(x, pa, 1, e.reshape(0, 4), pa[:0], 1, ids)
    torch.cuda.synchronize()


@pytest.mark.parametrize("N,nq,k,weights", [(3000, 70, 10, None), (40000, 5, 50, (1.0, 1e4)),
                                            (2500, 33, 7, "filter")])
def test_noalloc_matches_brute_force_twice(nhq, N, nq, k, weights):
    w = synth.int_valued(N, nq, 48, cards=(3, 4, 5), seed=N + nq)
    X, Qv = dev(w.X), dev(w.Qv)
    pa, pq = _packed(nhq, w.A), _packed(nhq, w.QA)
    ref_ids = torch.empty((nq, k), dtype=torch.uint32, device="cuda:0")
    ref_g = torch.empty((nq, k), dtype=torch.float32, device="cuda:0")
    ref_c = torch.empty((nq, k), dtype=torch.uint8, device="cuda:0")
    with nhq.Index.create(X, dev(w.A), weights if isinstance(weights, tuple) else None) as ix:
        nhq.nhq_brute_force(ix.handle, Qv, dev(w.QA), k, ref_ids, ref_g, ref_c,
                            weights="index" if weights is None else weights)
    torch.cuda.synchronize()
    outs = [(torch.full((nq, k), 7, dtype=torch.uint32, device="cuda:0"),
             torch.zeros((nq, k), dtype=torch.float32, device="cuda:0"),
             torch.zeros((nq, k), dtype=torch.uint8, device="cuda:0")) for _ in range(2)]
    free = []
    for ids, g, c in outs:  # two calls in a row share the fixed working array
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        nhq.nhq_brute_force_noalloc(X, pa, w.m, Qv, pq, k, ids, g, c, weights=weights)
        torch.cuda.synchronize()
        # integer components: every Gamma is exact, so the two entry points agree bit for bit
        assert (ids_i64(ids) == ids_i64(ref_ids)).all()
        assert torch.equal(c, ref_c)
        assert torch.equal(g, ref_g)
    # the second call allocated nothing on the device
    assert torch.cuda.mem_get_info()[0] == free[1]
    # and both equal the oracle's exact answer (integer components: Gamma exact in f32)
    O.build()
    ids = ids_i64(outs[1][0])
    if weights == "filter":
        want, dl, _ = O.filtered_topk(w.X, w.A, w.Qv, w.QA, k, prec=O.F32)
        assert (ids == want).all()
        g = outs[1][1].cpu().numpy().astype(np.float64)
        fin = want >= 0
        assert np.array_equal(g[fin], dl[fin])
    else:
        want, wg, wc = O.fused_topk(w.X, w.A, w.Qv, w.QA, k, weights=weights, prec=O.F32)
        assert (ids == want).all()
        assert np.array_equal(outs[1][1].cpu().numpy().astype(np.float64), wg)
        assert (outs[1][2].cpu().numpy().astype(np.int64) == wc).all()


def test_noalloc_refuses_a_batch_beyond_its_fixed_memory(nhq):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    N, d = 40000, 16
    big = next(((Q, k) for k in (256, 128) for Q in (2000, 1000, 500, 250)
                if _split_bytes(N, Q, k, sms) > FIXED_BYTES), None)
    if big is None:
        pytest.skip(f"with {sms} SMs every batch's split lists fit in the fixed array")
    Q, k = big
    w = synth.int_valued(N, Q, d, seed=5)
    X, Qv = dev(w.X), dev(w.Qv)
    pa, pq = _packed(nhq, w.A), _packed(nhq, w.QA)
    ids = torch.full((Q, k), 0xABCD, dtype=torch.uint32, device="cuda:0")
    with pytest.raises(nhq.NHQError) as e:
        nhq.nhq_brute_force_noalloc(X, pa, w.m, Qv, pq, k, ids)
    assert "scratch bytes" in str(e.value)
    torch.cuda.synchronize()
    assert (ids.cpu().numpy().astype(np.int64) == 0xABCD).all()  # nothing was written
    # the same batch in smaller pieces is accepted
    q2 = next(q for q in (100, 50, 25, 10) if _split_bytes(N, q, k, sms) <= FIXED_BYTES)
    small = torch.empty((q2, k), dtype=torch.uint32, device="cuda:0")
    nhq.nhq_brute_force_noalloc(X, pa, w.m, Qv[:q2].contiguous(), pq[:q2].contiguous(), k,
                                small)
    torch.cuda.synchronize()


def test_noalloc_refuses_the_weights_brute_force_refuses(nhq):
    # curve ii needs w_l = 0 or w_l >= 1, as in nhq_brute_force
    w = synth.int_valued(500, 4, 8, seed=6)
    X, Qv = dev(w.X), dev(w.Qv)
    pa, pq = _packed(nhq, w.A), _packed(nhq, w.QA)
    ids = torch.empty((4, 5), dtype=torch.uint32, device="cuda:0")
    for bad in (("harmonic", 0.5), (1.0, -1.0), (1.0, float("nan"))):
        with pytest.raises(nhq.NHQError):
            nhq.nhq_brute_force_noalloc(X, pa, w.m, Qv, pq, 5, ids, weights=bad)
