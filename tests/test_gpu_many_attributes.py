"""More than four attributes (the m = 6 and m = 9 settings of Sec. 6.4): the index packs
the m codes into one word with fields as narrow as the largest code allows, and every
kernel computes chi (Eq. 4-5) on those fields.  Each step is compared with the oracle,
which works on the byte codes directly, bit for bit on integer components; query codes
that no object has (above an attribute's largest code) must still count as mismatches."""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import dev, empty_out, ids_i64, to_u32_graph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CONST = (1.0, 10000.0)
CARDS6 = (3, 10, 20, 4, 5, 8)
CARDS9 = (3, 10, 20, 4, 5, 8, 2, 3, 6)  # 28 bits packed


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


def _unseen_codes(QA, cards):
    QA = QA.copy()
    QA[::5, 1] = 250              # above the largest code of attribute 1
    QA[1::7, len(cards) - 1] = 255
    return QA


@pytest.mark.parametrize("cards", [CARDS6, CARDS9])
@pytest.mark.parametrize("weights", [None, CONST])
def test_brute_force_exact(nhq, cards, weights):
    w = synth.int_valued(2500, 60, 40, cards=cards, seed=71)
    QA = _unseen_codes(w.QA, cards)
    ref_ids, ref_g, ref_chi = O.fused_topk(w.X, w.A, w.Qv, QA, 10, weights=weights, prec=O.F32)
    with nhq.Index.create(dev(w.X), dev(w.A), weights) as ix:
        assert ix.info[2] == len(cards)
        ids, g, chi = empty_out(w.nq, 10)
        nhq.nhq_brute_force(ix.handle, dev(w.Qv), dev(QA), 10, ids, g, chi)
        torch.cuda.synchronize()
    assert (ids_i64(ids) == ref_ids).all()
    assert (chi.cpu().numpy() == ref_chi).all()
    assert np.array_equal(g.cpu().numpy().astype(np.float64), ref_g)


@pytest.mark.parametrize("cards", [CARDS6, CARDS9])
@pytest.mark.parametrize("weights", [None, CONST])
def test_candidates_exact_f32_and_tensor_cores(nhq, cards, weights):
    w = synth.int_valued(2500, 1, 32, cards=cards, seed=72)
    ref, ref_g = O.knn(w.X, w.A, 64, weights=weights, prec=O.F32)
    with nhq.Index.create(dev(w.X), dev(w.A), weights) as ix:
        c32 = torch.empty((w.N, 64), dtype=torch.uint32, device="cuda:0")
        ctc = torch.empty((w.N, 64), dtype=torch.uint32, device="cuda:0")
        dtc = torch.empty((w.N, 64), dtype=torch.float32, device="cuda:0")
        nhq.nhq_knn(ix.handle, 64, c32)
        nhq.nhq_knn_bf16(ix.handle, 64, ctc, dtc)
        torch.cuda.synchronize()
    assert (ids_i64(c32) == ref).all()
    assert (ids_i64(ctc) == ref).all()
    assert np.array_equal(dtc.cpu().numpy().astype(np.float64), ref_g)


@pytest.mark.parametrize("knn_dtype", [0, 1])
def test_full_build_exact(nhq, knn_dtype):
    w = synth.int_valued(2200, 1, 32, cards=CARDS9, seed=73)
    ref, _, _ = O.build_graph(w.X, w.A, R=24, K=48, weights=CONST)
    with nhq.Index.build(dev(w.X), dev(w.A), degree=24, weights=CONST, K=48,
                         knn_dtype=knn_dtype) as ix:
        out = torch.empty((w.N, 24), dtype=torch.uint32, device="cuda:0")
        nhq.nhq_index_get_graph(ix.handle, out)
        torch.cuda.synchronize()
    assert (ids_i64(out) == ref).all()


@pytest.fixture(scope="module")
def graphs9():
    w = synth.int_valued(4000, 80, 32, cards=CARDS9, n_comp=20, seed=74)
    return w, {name: (wts, O.build_graph(w.X, w.A, R=16, K=32, weights=wts)[0])
               for name, wts in (("prop", None), ("const", CONST))}


@pytest.mark.parametrize("wname", ["prop", "const"])
@pytest.mark.parametrize("h", [1, 2])
@pytest.mark.parametrize("seed_mode", [0, 1, 3])
def test_search_exact(nhq, graphs9, wname, h, seed_mode):
    w, graphs = graphs9
    wts, nbr = graphs[wname]
    QA = _unseen_codes(w.QA, CARDS9)
    ref = O.search(w.X, w.A, nbr, w.Qv, QA, 10, 40, h=h, seed=13, weights=wts,
                   seed_mode=seed_mode)
    with nhq.Index.create(dev(w.X), dev(w.A), wts) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(QA), 10, 40, ids, g, chi, h=h, seed=13,
                       seed_mode=seed_mode)
        torch.cuda.synchronize()
    assert (ids_i64(ids) == ref["ids"]).all()
    assert (chi.cpu().numpy().astype(np.int32) == ref["chi"]).all()
    assert np.array_equal(g.cpu().numpy().astype(np.float64), ref["gamma"])


@pytest.mark.parametrize("entry", [0, 1])
def test_incremental_build_exact(nhq, entry):
    w = synth.int_valued(2001, 40, 32, cards=CARDS6, n_comp=20, seed=75)
    R, L, wave_max, cap = 16, 48, 128, 32
    ref = O.build_nsw(w.X, w.A, R=R, L=L, weights=CONST, seed=5, wave_max=wave_max,
                      rev_cap=cap, entry=entry)
    with nhq.Index.create(dev(w.X), dev(w.A), CONST) as ix:
        nhq.nhq_index_build_nsw(ix.handle, R, L=L, wave_max=wave_max, rev_cap=cap, seed=5,
                                entry=entry)
        g = torch.empty((w.N, R), dtype=torch.uint32, device="cuda:0")
        nhq.nhq_index_get_graph(ix.handle, g)
        torch.cuda.synchronize()
    assert (ids_i64(g) == ref).all()


def test_save_load_keeps_the_layout(nhq, graphs9, tmp_path):
    w, graphs = graphs9
    wts, nbr = graphs["const"]
    p = str(tmp_path / "ix9.nhq")
    QA = _unseen_codes(w.QA, CARDS9)
    with nhq.Index.create(dev(w.X), dev(w.A), wts) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        nhq.nhq_save(ix.handle, p)
        a = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(QA), 10, 40, *a, seed=3)
    with nhq.Index(nhq.nhq_load(p)) as ix2:
        assert ix2.info == (w.N, w.d, w.m, 16)
        b = empty_out(w.nq, 10)
        nhq.nhq_search(ix2.handle, dev(w.Qv), dev(QA), 10, 40, *b, seed=3)
        torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])


def test_attribute_limits(nhq):
    r = np.random.default_rng(1)
    X = r.integers(0, 255, (64, 8)).astype(np.float32)
    with pytest.raises(nhq.NHQError):      # 33 attributes
        nhq.Index.create(dev(X), dev(r.integers(0, 2, (64, 33)).astype(np.uint8)))
    A = r.integers(0, 256, (64, 5)).astype(np.uint8)
    A[0] = 255                             # 5 fields of 9 bits: more than 32
    with pytest.raises(nhq.NHQError):
        nhq.Index.create(dev(X), dev(A))
    A = r.integers(0, 2, (64, 16)).astype(np.uint8)   # 16 fields of 2 bits
    with nhq.Index.create(dev(X), dev(A)) as ix:
        assert ix.info[2] == 16
    with nhq.Index.create(dev(X), dev(np.zeros((64, 32), np.uint8))) as ix:  # 32 of 1 bit
        assert ix.info[2] == 32
