"""The incremental build (NPG_nsw of Sec. 4.3) in insertion waves: every wave searches
the graph of the vertices inserted before it, keeps a landing-zone selection and lets
the selected vertices re-select; waves see the graph as it was when they began, so the
build is deterministic and equals the oracle's bit for bit on integer components."""
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


@pytest.mark.parametrize("entry", [0, 1])
@pytest.mark.parametrize("weights", [None, CONST])
def test_incremental_build_matches_oracle(nhq, weights, entry):
    w = synth.int_valued(3001, 80, 32, cards=(3, 5, 7), n_comp=20, seed=97)
    R, L, wave_max, cap = 16, 48, 128, 32
    ref = O.build_nsw(w.X, w.A, R=R, L=L, weights=weights, seed=5, wave_max=wave_max,
                      rev_cap=cap, entry=entry)
    with nhq.Index.create(dev(w.X), dev(w.A), weights) as ix:
        nhq.nhq_index_build_nsw(ix.handle, R, L=L, wave_max=wave_max, rev_cap=cap, seed=5,
                                entry=entry)
        g = torch.empty((w.N, R), dtype=torch.uint32, device="cuda:0")
        nhq.nhq_index_get_graph(ix.handle, g)
        ids, gg, chi = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 48, ids, gg, chi, seed=2,
                       seed_mode=nhq.SEED_ATTRIBUTE)
        torch.cuda.synchronize()
    assert (ids_i64(g) == ref).all()
    sref = O.search(w.X, w.A, ref, w.Qv, w.QA, 10, 48, seed=2, weights=weights,
                    seed_mode=O.SEED_ATTRIBUTE)
    assert (ids_i64(ids) == sref["ids"]).all()
    assert np.array_equal(gg.cpu().numpy().astype(np.float64), sref["gamma"])
