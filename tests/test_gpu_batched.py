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
        wpq, wpb, bits, ms = nhq.nhq_autotune_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 64,
                                                     tmp, seed=1, seed_mode=nhq.SEED_ATTRIBUTE,
                                                     return_wpq=True)
        assert wpq in (1, 2, 4) and wpb in (2, 4, 8) and wpb % wpq == 0
        assert 8 <= bits <= 16 and ms > 0  # from the legal minimum (224 slots here)
        ids1, g1, c1 = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 64, ids1, g1, c1, seed=1,
                       seed_mode=nhq.SEED_ATTRIBUTE, warps_per_block=wpb, hash_bits=bits,
                       warps_per_query=wpq)
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


# ------------------------------------------------------------------ warps per query, beam width
@pytest.mark.parametrize("d", [32, 300])
@pytest.mark.parametrize("vec,rerank", [(0, 0), (1, 1), (2, 1)])
def test_warps_per_query_leave_results_unchanged(nhq, d, vec, rerank):
    # the helper warps only take distance passes: every output is the same for 1, 2, 4
    # warps per query (d = 300 takes the strided pass of wide rows)
    w = synth.int_valued(3000, 200, d, cards=(3, 5, 7), n_comp=20, seed=70 + d)
    nbr, _, _ = O.build_graph(w.X, w.A, R=16, K=32, weights=CONST)
    outs = []
    with nhq.Index.create(dev(w.X), dev(w.A), CONST) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        for wpq, wpb in ((1, 8), (2, 8), (4, 8), (2, 2), (4, 4)):
            for h, sm in ((1, nhq.SEED_ATTRIBUTE), (2, nhq.SEED_RANDOM)):
                ids, g, c = empty_out(w.nq, 10)
                ndc = torch.empty(w.nq, dtype=torch.int32, device="cuda:0")
                ex = torch.empty(w.nq, dtype=torch.int32, device="cuda:0")
                nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 40, ids, g, c, ndc=ndc,
                               expansions=ex, h=h, seed=3, seed_mode=sm, vec_dtype=vec,
                               rerank=rerank, warps_per_query=wpq, warps_per_block=wpb)
                torch.cuda.synchronize()
                outs.append(((wpq, wpb, h), [t.cpu() for t in (ids, g, c, ndc, ex)]))
    ref = {key[2]: o for key, o in outs if key[0] == 1}
    for key, o in outs:
        for a, b in zip(o, ref[key[2]]):
            assert torch.equal(a, b), key
    # and the 4-warp form against the oracle directly
    r = O.search(w.X, w.A, nbr, w.Qv, w.QA, 10, 40, seed=3, weights=CONST,
                 seed_mode=O.SEED_ATTRIBUTE, vec_round=vec, rerank=bool(rerank))
    four = dict(outs)[(4, 8, 1)]
    assert (ids_i64(four[0]) == r["ids"]).all()
    assert np.array_equal(four[1].numpy().astype(np.float64), r["gamma"])


def test_warps_per_query_rejects_bad_values(nhq, case):
    w, nbr = case
    with nhq.Index.create(dev(w.X), dev(w.A), CONST) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, c = empty_out(w.nq, 10)
        for wpq, wpb in ((3, 0), (8, 0), (4, 2)):
            with pytest.raises(nhq.NHQError):
                nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 40, ids, g, c,
                               warps_per_query=wpq, warps_per_block=wpb)


def test_recall_matches_the_oracle_definition(nhq, case):
    w, nbr = case
    truth, _, P = O.filtered_topk(w.X, w.A, w.Qv, w.QA, 10, prec=O.F32)
    with nhq.Index.create(dev(w.X), dev(w.A), CONST) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        for ef in (10, 20, 80):
            ids, g, c = empty_out(w.nq, 10)
            nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, ef, ids, g, c, seed=2)
            r = nhq.nhq_recall(ids, dev(to_u32_graph(truth)))
            want, _ = O.hybrid_recall(ids_i64(ids), w.A, w.QA, truth, P)
            assert abs(r - want) < 1e-6, (ef, r, want)


def test_autotune_beam_takes_the_smallest_ef_reaching_the_target(nhq, case):
    w, nbr = case
    truth, _, P = O.filtered_topk(w.X, w.A, w.Qv, w.QA, 10, prec=O.F32)
    efs = [10, 12, 16, 24, 32, 48, 64, 128]
    with nhq.Index.create(dev(w.X), dev(w.A), CONST) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        rec = {}
        for ef in efs:
            ids, g, c = empty_out(w.nq, 10)
            nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, ef, ids, g, c, seed=2,
                           seed_mode=nhq.SEED_ATTRIBUTE)
            rec[ef] = O.hybrid_recall(ids_i64(ids), w.A, w.QA, truth, P)[0]
        target = 0.97
        want = next((e for e in efs if rec[e] >= target), efs[-1])
        tmp = torch.empty((w.nq, 10), dtype=torch.uint32, device="cuda:0")
        t = nhq.nhq_autotune_beam(ix.handle, dev(w.Qv), dev(w.QA), 10, efs,
                                  dev(to_u32_graph(truth)), target, tmp, seed=2,
                                  seed_mode=nhq.SEED_ATTRIBUTE)
    assert t["ef"] == want, (t, rec)
    assert abs(t["recall"] - rec[want]) < 1e-6
    assert t["warps_per_query"] in (1, 2, 4) and t["warps_per_block"] in (2, 4, 8)
    assert t["warps_per_block"] % t["warps_per_query"] == 0 and t["ms"] > 0


@pytest.mark.parametrize("d", [32, 64, 128])
@pytest.mark.parametrize("vec", [0, 1])
def test_tile_rows_leave_results_unchanged(nhq, d, vec):
    # four rows per team and pass (one pass for a typical expansion) against two: on
    # integer components every sum is exact, so every output is the same; d = 32, 64 and
    # 128 take the three fixed-chunk forms of the f32 rows
    w = synth.int_valued(3000, 200, d, cards=(3, 5, 7), n_comp=20, seed=90 + d)
    nbr, _, _ = O.build_graph(w.X, w.A, R=16, K=32, weights=CONST)
    outs = {}
    with nhq.Index.create(dev(w.X), dev(w.A), CONST) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        for tr, wpq in ((2, 1), (2, 2), (4, 1)):
            if True:
                ids, g, c = empty_out(w.nq, 10)
                ndc = torch.empty(w.nq, dtype=torch.int32, device="cuda:0")
                nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 48, ids, g, c, ndc=ndc,
                               seed=3, seed_mode=nhq.SEED_ATTRIBUTE, vec_dtype=vec,
                               tile_rows=tr, warps_per_query=wpq)
                torch.cuda.synchronize()
                outs[(tr, wpq)] = [t.cpu() for t in (ids, g, c, ndc)]
        for bad in (dict(tile_rows=3), dict(tile_rows=4, warps_per_query=2)):
            with pytest.raises(nhq.NHQError):
                nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 48, ids, g, c, **bad)
    for key, o in outs.items():
        for a, b in zip(o, outs[(2, 1)]):
            assert torch.equal(a, b), key
    r = O.search(w.X, w.A, nbr, w.Qv, w.QA, 10, 48, seed=3, weights=CONST,
                 seed_mode=O.SEED_ATTRIBUTE, vec_round=vec)
    assert (ids_i64(outs[(4, 1)][0]) == r["ids"]).all()


def test_batched_tuner_and_captured_batched_search(nhq, case):
    # a heterogeneous batch: the tuned shape and the captured launch return what the
    # plain batched call returns, and the graph replays after its inputs change in place
    w, nbr = case
    k_arr, ef_arr = synth.mixed_k_ef(w.nq, seed=95, ks=(1, 5, 10), ef_lo=12, ef_hi=80)
    kmax = 10
    with nhq.Index.create(dev(w.X), dev(w.A), CONST) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        kd, efd = dev(k_arr), dev(ef_arr)
        ref, refg, _ = empty_out(w.nq, kmax)
        nhq.nhq_search_batched(ix.handle, dev(w.Qv), dev(w.QA), kd, efd, kmax, ref, refg,
                               seed=4, seed_mode=nhq.SEED_ATTRIBUTE)
        tmp = torch.empty((w.nq, kmax), dtype=torch.uint32, device="cuda:0")
        t = nhq.nhq_autotune_batched(ix.handle, dev(w.Qv), dev(w.QA), kd, efd, kmax, tmp,
                                     seed=4, seed_mode=nhq.SEED_ATTRIBUTE)
        assert t["warps_per_query"] in (1, 2, 4) and t["tile_rows"] in (2, 4) and t["ms"] > 0
        shape = {x: t[x] for x in ("warps_per_query", "tile_rows", "warps_per_block",
                                   "hash_bits")}
        ids, g, _ = empty_out(w.nq, kmax)
        nhq.nhq_search_batched(ix.handle, dev(w.Qv), dev(w.QA), kd, efd, kmax, ids, g, seed=4,
                               seed_mode=nhq.SEED_ATTRIBUTE, **shape)
        torch.cuda.synchronize()
        assert torch.equal(ids, ref) and torch.equal(g, refg)
        Qd, QAd = dev(w.Qv), dev(w.QA)
        gids, gg, _ = empty_out(w.nq, kmax)
        graph = nhq.nhq_search_graph_create_batched(ix.handle, Qd, QAd, kd, efd, kmax, gids,
                                                    gg, seed=4, seed_mode=nhq.SEED_ATTRIBUTE)
        gids.fill_(0)
        graph.launch()
        torch.cuda.synchronize()
        assert torch.equal(gids, ref) and torch.equal(gg, refg)
        # new queries written in place, replayed
        Qd.copy_(torch.flip(Qd, [0]))
        QAd.copy_(torch.flip(QAd, [0]))
        graph.launch()
        ref2, refg2, _ = empty_out(w.nq, kmax)
        nhq.nhq_search_batched(ix.handle, Qd, QAd, kd, efd, kmax, ref2, refg2, seed=4,
                               seed_mode=nhq.SEED_ATTRIBUTE)
        torch.cuda.synchronize()
        graph.close()
        assert torch.equal(gids, ref2) and torch.equal(gg, refg2)
