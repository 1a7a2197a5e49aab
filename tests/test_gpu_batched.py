"""Batched form: the autotuner, captured search graphs and a heterogeneous
batch on cluster-correlated attributes (mixed k and ef in one launch)."""
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


@pytest.fixture(scope="module")
def case():
    w = synth.int_valued(5000, 300, 32, cards=(3, 5, 7), n_comp=20, seed=51)
    nbr, _, _ = O.build_graph(w.X, w.A, R=16, K=32, weights=CONST)
    return w, nbr


def test_autotune_keeps_results_and_returns_a_legal_shape(nhq, case):
    w, nbr = case
    with nhq.Index.create(dev(w.X), dev(w.A), CONST) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids0, g0, c0 = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 64, ids0, g0, c0, seed=1,
                       seed_mode=nhq.SEED_ATTRIBUTE)
        tmp = torch.empty((w.nq, 10), dtype=torch.uint32, device="cuda:0")
        wpb, bits, ms = nhq.nhq_autotune_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 64, tmp,
                                                seed=1, seed_mode=nhq.SEED_ATTRIBUTE)
        assert wpb in (2, 4, 8) and 10 <= bits <= 16 and ms > 0
        ids1, g1, c1 = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 64, ids1, g1, c1, seed=1,
                       seed_mode=nhq.SEED_ATTRIBUTE, warps_per_block=wpb, hash_bits=bits)
        torch.cuda.synchronize()
    assert torch.equal(ids0, ids1) and torch.equal(g0, g1)


def test_captured_graph_replays_the_search(nhq, case):
    w, nbr = case
    half = w.nq // 2
    with nhq.Index.create(dev(w.X), dev(w.A), CONST) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        Qb, QAb = dev(w.Qv[:half]), dev(w.QA[:half])
        ids, g, chi = empty_out(half, 10)
        graph = nhq.SearchGraph(ix.handle, Qb, QAb, 10, 40, ids, g, chi, seed=4,
                                seed_mode=nhq.SEED_ATTRIBUTE, vec_dtype=nhq.VEC_BF16)
        for part in (slice(0, half), slice(half, 2 * half)):
            Qb.copy_(dev(w.Qv[part]))
            QAb.copy_(dev(w.QA[part]))
            ids.zero_()
            graph.launch()
            ref_ids, ref_g, ref_c = empty_out(half, 10)
            nhq.nhq_search(ix.handle, Qb, QAb, 10, 40, ref_ids, ref_g, ref_c, seed=4,
                           seed_mode=nhq.SEED_ATTRIBUTE, vec_dtype=nhq.VEC_BF16)
            torch.cuda.synchronize()
            assert torch.equal(ids, ref_ids) and torch.equal(g, ref_g)
        graph.close()


def test_heterogeneous_batch_on_correlated_attributes(nhq):
    w = synth.c4(N=6000, nq=400, d=32, n_comp=30, seed=52)
    nbr, _, _ = O.build_graph(w.X, w.A, R=16, K=32, weights=CONST)
    k_arr, ef_arr = synth.mixed_k_ef(w.nq, seed=53, ks=(1, 10, 100), ef_lo=16, ef_hi=512)
    k_max = int(k_arr.max())
    with nhq.Index.create(dev(w.X), dev(w.A), CONST) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, k_max)
        st = torch.empty(w.nq, dtype=torch.int32, device="cuda:0")
        nhq.nhq_search_batched(ix.handle, dev(w.Qv), dev(w.QA), dev(k_arr), dev(ef_arr), k_max,
                               ids, g, chi, st, seed=3, seed_mode=nhq.SEED_ATTRIBUTE)
        torch.cuda.synchronize()
    got = ids_i64(ids)
    assert (st.cpu().numpy() == 0).all()
    # float data: compare with the oracle row by row on a sample, values to 1e-5 and
    # ids up to near-ties (at most a few swapped positions in total)
    rows = np.random.default_rng(0).choice(w.nq, 40, replace=False)
    swaps = 0
    for q in rows:
        r = O.search(w.X, w.A, nbr, w.Qv[:q + 1], w.QA[:q + 1], int(k_arr[q]), int(ef_arr[q]),
                     seed=3, weights=CONST, seed_mode=O.SEED_ATTRIBUTE)
        kq = int(k_arr[q])
        assert np.allclose(g.cpu().numpy()[q, :kq], r["gamma"][q], rtol=1e-5, atol=0)
        swaps += int((got[q, :kq] != r["ids"][q]).sum())
        assert (got[q, kq:] == -1).all()
    assert swaps <= 4
