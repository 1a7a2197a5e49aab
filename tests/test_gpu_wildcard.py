"""Partial attribute constraints: with the wildcard switch on, a query code 255 leaves its
attribute unconstrained (it never counts toward chi, and under the attribute seed modes an
open query takes its seeds from the runs of its completions, or the random stream when it
has more than 64).  The paper's hybrid query constrains every attribute, so this is an
extension; every result is compared with the oracle's reading of it, bit for bit on
integer components, for the byte layout (m = 3) and for bit fields (m = 6, 9)."""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import dev, empty_out, ids_i64, to_u32_graph

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


def _open(QA):
    QA = QA.copy()
    m = QA.shape[1]
    QA[::3, 0] = 255                  # one open position
    QA[1::4, m - 1] = 255             # another (some queries have both)
    QA[::11, :] = 255                 # fully open: plain L2
    return QA


@pytest.mark.parametrize("cards", [(3, 10, 20), (3, 10, 20, 4, 5, 8)])
@pytest.mark.parametrize("weights", [None, CONST])
def test_brute_force_with_open_positions(nhq, cards, weights):
    w = synth.int_valued(2500, 66, 40, cards=cards, seed=81)
    QA = _open(w.QA)
    ref_ids, ref_g, ref_chi = O.fused_topk(w.X, w.A, w.Qv, QA, 10, weights=weights, prec=O.F32,
                                           wildcard=255)
    with nhq.Index.create(dev(w.X), dev(w.A), weights) as ix:
        ids, g, chi = empty_out(w.nq, 10)
        nhq.nhq_brute_force(ix.handle, dev(w.Qv), dev(QA), 10, ids, g, chi, wildcard=1)
        torch.cuda.synchronize()
    assert (ids_i64(ids) == ref_ids).all()
    assert (chi.cpu().numpy() == ref_chi).all()
    assert np.array_equal(g.cpu().numpy().astype(np.float64), ref_g)


@pytest.mark.parametrize("cards", [(3, 10, 20), (3, 10, 20, 4, 5, 8)])
def test_filter_mode_ground_truth_with_open_positions(nhq, cards):
    w = synth.int_valued(3000, 50, 16, cards=cards, seed=82)
    QA = _open(w.QA)
    ref_ids, _, P = O.filtered_topk(w.X, w.A, w.Qv, QA, 10, prec=O.F32, wildcard=255)
    with nhq.Index.create(dev(w.X), dev(w.A)) as ix:
        ids, g, chi = empty_out(w.nq, 10)
        nhq.nhq_brute_force(ix.handle, dev(w.Qv), dev(QA), 10, ids, g, chi, weights="filter",
                            wildcard=1)
        torch.cuda.synchronize()
    got = ids_i64(ids)
    gi = g.cpu().numpy()
    for q in range(w.nq):
        n = min(10, int(P[q]))
        assert (got[q, :n] == ref_ids[q, :n]).all(), q
        assert np.isinf(gi[q, n:]).all()


@pytest.fixture(scope="module")
def graphs():
    out = {}
    for cards in ((3, 5, 7), (3, 10, 20, 4, 5, 8, 2, 3, 6)):
        w = synth.int_valued(4000, 72, 32, cards=cards, n_comp=20, seed=83)
        out[len(cards)] = (w, {name: (wts, O.build_graph(w.X, w.A, R=16, K=32, weights=wts)[0])
                               for name, wts in (("prop", None), ("const", CONST))})
    return out


@pytest.mark.parametrize("m", [3, 9])
@pytest.mark.parametrize("wname", ["prop", "const"])
@pytest.mark.parametrize("seed_mode", [0, 1, 3])
def test_search_with_open_positions(nhq, graphs, m, wname, seed_mode):
    w, gs = graphs[m]
    wts, nbr = gs[wname]
    QA = _open(w.QA)
    ref = O.search(w.X, w.A, nbr, w.Qv, QA, 10, 40, seed=17, weights=wts, seed_mode=seed_mode,
                   wildcard=255)
    with nhq.Index.create(dev(w.X), dev(w.A), wts) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(QA), 10, 40, ids, g, chi, seed=17,
                       seed_mode=seed_mode, wildcard=1)
        torch.cuda.synchronize()
    assert (ids_i64(ids) == ref["ids"]).all()
    assert (chi.cpu().numpy().astype(np.int32) == ref["chi"]).all()
    assert np.array_equal(g.cpu().numpy().astype(np.float64), ref["gamma"])


def test_wildcard_off_keeps_255_an_ordinary_code(nhq, graphs):
    w, gs = graphs[3]
    wts, nbr = gs["const"]
    QA = _open(w.QA)
    ref = O.search(w.X, w.A, nbr, w.Qv, QA, 10, 40, seed=17, weights=wts)
    with nhq.Index.create(dev(w.X), dev(w.A), wts) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(QA), 10, 40, ids, g, chi, seed=17)
        with pytest.raises(nhq.NHQError):
            nhq.nhq_search(ix.handle, dev(w.Qv), dev(QA), 10, 40, ids, g, chi, wildcard=2)
        torch.cuda.synchronize()
    assert (ids_i64(ids) == ref["ids"]).all()
    assert (chi.cpu().numpy().astype(np.int32) == ref["chi"]).all()


@pytest.mark.parametrize("seed_mode", [1, 3])
def test_search_open_queries_with_many_completions(nhq, graphs, seed_mode):
    # attributes 1 and 2 open: 5 x 7 = 35 completions (more than one per lane), and runs
    # of about 1,300 members, so the nearest rule samples 256 of them
    w, gs = graphs[3]
    wts, nbr = gs["const"]
    QA = w.QA.copy()
    QA[::2, 1:] = 255
    ref = O.search(w.X, w.A, nbr, w.Qv, QA, 10, 40, seed=19, weights=wts, seed_mode=seed_mode,
                   wildcard=255)
    with nhq.Index.create(dev(w.X), dev(w.A), wts) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(QA), 10, 40, ids, g, chi, seed=19,
                       seed_mode=seed_mode, wildcard=1)
        torch.cuda.synchronize()
    assert (ids_i64(ids) == ref["ids"]).all()
    assert np.array_equal(g.cpu().numpy().astype(np.float64), ref["gamma"])
