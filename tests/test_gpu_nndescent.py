"""Candidate sets by NN-descent (Sec. 4.3, the NPG_kgraph recipe): the lists are
approximate and their update order races, so they are checked by what must hold for
any run: graph quality (Eq. 7) against the exact candidate sets, rows sorted by
(Gamma, id) without the vertex itself or repeats, every Gamma equal to the oracle's f32
value (integer components make it exact), and a composite index built on them
searching nearly as well as one built on the exact sets."""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import dev, empty_out, ids_i64

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CONST = (1.0, 10000.0)


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


@pytest.mark.parametrize("weights", [None, CONST])
def test_nndescent_lists(nhq, weights):
    w = synth.int_valued(20000, 1, 32, seed=90)
    K = 32
    with nhq.Index.create(dev(w.X), dev(w.A), weights) as ix:
        ids = torch.empty((w.N, K), dtype=torch.uint32, device="cuda:0")
        g = torch.empty((w.N, K), dtype=torch.float32, device="cuda:0")
        iters = nhq.nhq_knn_nndescent(ix.handle, K, ids, g)
        ex = torch.empty((w.N, K), dtype=torch.uint32, device="cuda:0")
        nhq.nhq_knn(ix.handle, K, ex)
        torch.cuda.synchronize()
    got, gg, exact = ids_i64(ids), g.cpu().numpy().astype(np.float64), ids_i64(ex)
    assert 1 <= iters <= 12
    quality = O.graph_quality(got, exact)
    print(f"weights {weights}: {iters} iterations, graph quality {quality:.4f}")
    assert quality >= 0.9
    u = np.arange(w.N)[:, None]
    assert ((got >= 0) & (got < w.N)).all() and not (got == u).any()
    for r in range(0, w.N, 97):
        assert len(set(got[r].tolist())) == K
        keys = list(zip(gg[r], got[r]))
        assert keys == sorted(keys)
        want = [O.gamma(O.delta(w.X[r], w.X[v], O.F32), O.chi(w.A[r], w.A[v]), w.m, weights,
                        O.F32) for v in got[r]]
        assert np.array_equal(gg[r], np.array(want))


def test_index_on_nndescent_candidates_searches_well(nhq):
    w = synth.int_valued(20000, 400, 32, cards=(3, 5, 7), n_comp=40, seed=91)
    out = {}
    for dtype in (0, 2):
        with nhq.Index.build(dev(w.X), dev(w.A), degree=24, weights=CONST, K=48,
                             knn_dtype=dtype) as ix:
            ids, g, chi = empty_out(w.nq, 10)
            nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 48, ids, g, chi, seed=3,
                           seed_mode=nhq.SEED_ATTRIBUTE)
            torch.cuda.synchronize()
            out[dtype] = ids_i64(ids)
    truth = O.fused_topk(w.X, w.A, w.Qv, w.QA, 10, weights=CONST, prec=O.F32)[0]
    rec = {d: np.mean([len(set(a) & set(b)) / 10 for a, b in zip(out[d], truth)]) for d in out}
    print(f"Gamma-recall@10: exact candidates {rec[0]:.4f}, NN-descent {rec[2]:.4f}")
    assert rec[2] >= rec[0] - 0.02
