"""Typed vector input at the boundary (nhq_index_create_typed / nhq_build_typed): f16 and
bf16 rows are widened to f32 exactly and also kept as the index's scoring copy of their
type, so a search that scores with that copy reads 2 d bytes per row and returns what
the f32 search returns on the same values."""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import assert_topk_near_tie_equal, dev, empty_out, ids_i64, to_u32_graph

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


@pytest.mark.parametrize("tdt,vec", [("float16", 3), ("bfloat16", 1)])
def test_typed_input_scores_like_f32(nhq, tdt, vec):
    # integer components 0..255 are exact in f16 and bf16
    w = synth.int_valued(3000, 120, 40, cards=(3, 5, 7), n_comp=20, seed=91)
    nbr, _, _ = O.build_graph(w.X, w.A, R=16, K=32, weights=CONST)
    Xt = torch.from_numpy(w.X).to("cuda:0").to(getattr(torch, tdt))
    outs = []
    for X, v in ((dev(w.X), 0), (Xt, vec)):
        with nhq.Index.create(X, dev(w.A), CONST) as ix:
            nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
            ids, g, c = empty_out(w.nq, 10)
            nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 40, ids, g, c, seed=4,
                           vec_dtype=v, seed_mode=nhq.SEED_ATTRIBUTE)
            torch.cuda.synchronize()
            outs.append((ids.cpu(), g.cpu(), c.cpu()))
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    r = O.search(w.X, w.A, nbr, w.Qv, w.QA, 10, 40, seed=4, weights=CONST,
                 seed_mode=O.SEED_ATTRIBUTE)
    assert (ids_i64(outs[1][0]) == r["ids"]).all()


def test_typed_build_from_f16_matches_the_oracle(nhq):
    # c5-shaped float rows (every value an f16): the typed build and f16 scoring against
    # the oracle's build and search on the same values
    w = synth.c5(N=4000, nq=60, d=96, cards=(4, 5, 6), n_comp=40, seed=92)
    ref_nbr, _, _ = O.build_graph(w.X, w.A, R=16, K=32, weights=CONST, prec=O.F32)
    X16 = torch.from_numpy(w.X.astype(np.float16)).to("cuda:0")
    with nhq.Index.build(X16, dev(w.A), degree=16, weights=CONST, K=32) as ix:
        out = torch.empty((w.N, 16), dtype=torch.uint32, device="cuda:0")
        nhq.nhq_index_get_graph(ix.handle, out)
        ids, g, c = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 48, ids, g, c, seed=6,
                       vec_dtype=nhq.VEC_F16, seed_mode=nhq.SEED_ATTRIBUTE)
        torch.cuda.synchronize()
    # the build on float rows matches up to near-ties of the f32 sums: most rows agree
    same = (ids_i64(out) == ref_nbr).all(axis=1).mean()
    assert same > 0.5, same
    r = O.search(w.X, w.A, ids_i64(out), w.Qv, w.QA, 10, 48, seed=6, weights=CONST,
                 seed_mode=O.SEED_ATTRIBUTE, vec_round=O.ROUND_F16)
    assert_topk_near_tie_equal(O, w.X, w.A, w.Qv, w.QA, ids_i64(ids),
                               g.cpu().numpy().astype(np.float64), r["ids"], r["gamma"], CONST)


def test_typed_input_rejects_non_finite_values(nhq):
    w = synth.int_valued(200, 1, 8, seed=93)
    X = torch.from_numpy(w.X).to(torch.float16).to("cuda:0")
    X[7, 3] = float("inf")
    with pytest.raises(nhq.NHQError):
        nhq.Index.create(X, dev(w.A), CONST)
