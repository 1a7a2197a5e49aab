"""The harmonic weightings of Sec. 6.5 (curve i: Gamma = 2 delta chi / (delta + chi);
curve ii: chi replaced by 1 / c chi, c = 100) through every kernel, bit for bit against
the oracle on integer components: brute force, exact candidate sets on f32 and on the
tensor cores, the whole build, and the search."""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import dev, empty_out, ids_i64, to_u32_graph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CURVES = ["harmonic", ("harmonic", 100.0)]


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


@pytest.fixture(scope="module")
def data():
    return synth.int_valued(2000, 60, 32, cards=(3, 5, 7), n_comp=16, seed=95)


@pytest.mark.parametrize("weights", CURVES)
def test_brute_force(nhq, data, weights):
    w = data
    with nhq.Index.create(dev(w.X), dev(w.A), weights) as ix:
        ids, g, chi = empty_out(w.nq, 10)
        nhq.nhq_brute_force(ix.handle, dev(w.Qv), dev(w.QA), 10, ids, g, chi)
        torch.cuda.synchronize()
    ref_i, ref_g, ref_c = O.fused_topk(w.X, w.A, w.Qv, w.QA, 10, weights=weights, prec=O.F32)
    assert (ids_i64(ids) == ref_i).all()
    assert np.array_equal(g.cpu().numpy().astype(np.float64), ref_g)


@pytest.mark.parametrize("weights", CURVES)
def test_candidates_f32_and_tensor_cores(nhq, data, weights):
    w = data
    ref, ref_g = O.knn(w.X, w.A, 48, weights=weights, prec=O.F32)
    with nhq.Index.create(dev(w.X), dev(w.A), weights) as ix:
        for fn in (nhq.nhq_knn, nhq.nhq_knn_bf16):
            cand = torch.empty((w.N, 48), dtype=torch.uint32, device="cuda:0")
            dist = torch.empty((w.N, 48), dtype=torch.float32, device="cuda:0")
            fn(ix.handle, 48, cand, dist)
            torch.cuda.synchronize()
            assert (ids_i64(cand) == ref).all(), fn.__name__
            assert np.array_equal(dist.cpu().numpy().astype(np.float64), ref_g), fn.__name__


@pytest.mark.parametrize("weights", CURVES)
def test_build_and_search(nhq, data, weights):
    w = data
    ref_nbr, _, _ = O.build_graph(w.X, w.A, R=16, K=32, weights=weights)
    with nhq.Index.build(dev(w.X), dev(w.A), degree=16, weights=weights, K=32,
                         knn_dtype=1) as ix:
        g = torch.empty((w.N, 16), dtype=torch.uint32, device="cuda:0")
        nhq.nhq_index_get_graph(ix.handle, g)
        ids, gg, chi = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 48, ids, gg, chi, seed=6,
                       seed_mode=nhq.SEED_ATTRIBUTE)
        torch.cuda.synchronize()
    assert (ids_i64(g) == ref_nbr).all()
    ref = O.search(w.X, w.A, ref_nbr, w.Qv, w.QA, 10, 48, seed=6, weights=weights,
                   seed_mode=O.SEED_ATTRIBUTE)
    assert (ids_i64(ids) == ref["ids"]).all()
    assert np.array_equal(gg.cpu().numpy().astype(np.float64), ref["gamma"])
    assert (chi.cpu().numpy() == ref["chi"]).all()
