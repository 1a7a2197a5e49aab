"""The strategies the paper compares NHQ against, built from this library's kernels:
post-filtering (a proximity graph on vector distance only, searched for k' records,
then the records whose attributes match) and pre-filtering (exact top-k among the
matching objects, the filter-mode brute force)."""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import dev, empty_out, ids_i64, to_u32_graph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L2 = (1.0, 0.0)  # constant weights with w_l = 0: Gamma = delta, a plain L2 graph


@pytest.fixture(scope="module")
def nhq():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2203_13601_gb300 import build as B

    B.build()
    O.build()
    import paper_2203_13601_gb300 as m

    m.load_library()
    return m


def _keep_matching(ids, dists, chi, k):
    out_i = np.full((ids.shape[0], k), -1, np.int64)
    out_d = np.full((ids.shape[0], k), np.inf)
    for q in range(ids.shape[0]):
        sel = np.nonzero((ids[q] >= 0) & (chi[q] == 0))[0][:k]
        out_i[q, :len(sel)] = ids[q, sel]
        out_d[q, :len(sel)] = dists[q, sel]
    return out_i, out_d


def test_postfilter_search_on_an_l2_graph(nhq):
    w = synth.int_valued(4000, 120, 32, cards=(3, 5, 7), n_comp=20, seed=81)
    nbr, _, _ = O.build_graph(w.X, w.A, R=16, K=32, weights=L2)
    kp, k = 64, 10
    with nhq.Index.create(dev(w.X), dev(w.A), L2) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, kp)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), kp, 96, ids, g, chi, seed=4)
        fi = torch.empty((w.nq, k), dtype=torch.uint32, device="cuda:0")
        fd = torch.empty((w.nq, k), dtype=torch.float32, device="cuda:0")
        nhq.nhq_postfilter(ids, g, chi, k, fi, fd)
        torch.cuda.synchronize()
    # the search on the L2 graph is the oracle's; its post-filter keeps the matches in order
    ref = O.search(w.X, w.A, nbr, w.Qv, w.QA, kp, 96, seed=4, weights=L2)
    assert (ids_i64(ids) == ref["ids"]).all()
    assert (chi.cpu().numpy() == ref["chi"]).all()
    want_i, want_d = _keep_matching(ref["ids"], ref["gamma"], ref["chi"], k)
    assert (ids_i64(fi) == want_i).all()
    assert np.array_equal(fd.cpu().numpy().astype(np.float64), want_d)


def test_postfilter_pads_and_accepts_host_arrays(nhq):
    ids = np.array([[5, 7, 9, 0xFFFFFFFF], [1, 2, 3, 4]], np.uint32)
    d = np.array([[0.1, 0.2, 0.3, np.inf], [1, 2, 3, 4]], np.float32)
    chi = np.array([[0, 1, 0, 255], [1, 1, 1, 0]], np.uint8)
    oi = np.empty((2, 3), np.uint32)
    od = np.empty((2, 3), np.float32)
    nhq.nhq_postfilter(ids, d, chi, 3, oi, od)
    assert oi.tolist() == [[5, 9, 0xFFFFFFFF], [4, 0xFFFFFFFF, 0xFFFFFFFF]]
    assert od[0, 0] == np.float32(0.1) and od[1, 0] == 4 and np.isinf(od[0, 2])
