"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer-valued workloads make every squared distance an integer below 2^24, so
f32 evaluation is exact in any order: ids, chi and Gamma must then match the
oracle's canonical-f32 results bit for bit.  Float workloads are compared with
values within 1e-5 relative of the f64 oracle and ids equal up to near-ties.
"""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import (NONE, assert_topk_near_tie_equal, dev, empty_out, ids_i64,
                     to_u32_graph)

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


def _index(nhq, w, weights=None):
    return nhq.Index.create(dev(w.X), dev(w.A), weights)


# ------------------------------------------------------------------ brute force (Def. 2)
@pytest.mark.parametrize("weights", [None, CONST])
@pytest.mark.parametrize("k", [1, 10, 100])
def test_brute_force_exact_on_integer_data(nhq, weights, k):
    w = synth.int_valued(3000, 70, 48, cards=(3, 4, 5), seed=31)  # ragged N, Q, d tiles
    ref_ids, ref_g, ref_chi = O.fused_topk(w.X, w.A, w.Qv, w.QA, k, weights=weights, prec=O.F32)
    with _index(nhq, w, weights) as ix:
        ids, g, chi = empty_out(w.nq, k)
        nhq.nhq_brute_force(ix.handle, dev(w.Qv), dev(w.QA), k, ids, g, chi)
        torch.cuda.synchronize()
    assert (ids_i64(ids) == ref_ids).all()
    assert (chi.cpu().numpy() == ref_chi).all()
    assert np.array_equal(g.cpu().numpy().astype(np.float64), ref_g)


def test_brute_force_filter_mode_is_hybrid_ground_truth(nhq):
    w = synth.int_valued(4000, 50, 16, cards=(3, 10, 20), seed=32)
    ref_ids, ref_dl, P = O.filtered_topk(w.X, w.A, w.Qv, w.QA, 10, prec=O.F32)
    with _index(nhq, w) as ix:
        ids, g, chi = empty_out(w.nq, 10)
        nhq.nhq_brute_force(ix.handle, dev(w.Qv), dev(w.QA), 10, ids, g, chi, weights="filter")
        torch.cuda.synchronize()
    got = ids_i64(ids)
    assert (got == ref_ids).all()
    gg = g.cpu().numpy().astype(np.float64)
    assert np.array_equal(gg[np.isfinite(ref_dl)], ref_dl[np.isfinite(ref_dl)])
    assert (P < 10).any()  # some queries have fewer matches than k: padded rows checked


def test_brute_force_float_data_near_ties(nhq):
    w = synth.c1(N=5000, nq=40, d=100, seed=33)
    ref_ids, ref_g, _ = O.fused_topk(w.X, w.A, w.Qv, w.QA, 10)
    with _index(nhq, w) as ix:
        ids, g, chi = empty_out(w.nq, 10)
        nhq.nhq_brute_force(ix.handle, dev(w.Qv), dev(w.QA), 10, ids, g, chi)
        torch.cuda.synchronize()
    swaps = assert_topk_near_tie_equal(O, w.X, w.A, w.Qv, w.QA, ids_i64(ids), g.cpu().numpy(),
                                       ref_ids, ref_g, None)
    assert swaps <= 4


def test_brute_force_split_and_merge(nhq):
    # few queries over many objects: the object range is split and the lists merged
    w = synth.int_valued(40000, 3, 16, seed=34)
    ref_ids, ref_g, _ = O.fused_topk(w.X, w.A, w.Qv, w.QA, 50, prec=O.F32)
    with _index(nhq, w) as ix:
        ids, g, chi = empty_out(w.nq, 50)
        nhq.nhq_brute_force(ix.handle, dev(w.Qv), dev(w.QA), 50, ids, g, chi)
        torch.cuda.synchronize()
    assert (ids_i64(ids) == ref_ids).all()


def test_brute_force_k_larger_than_N(nhq):
    w = synth.int_valued(20, 5, 8, seed=35)
    ref_ids, _, _ = O.fused_topk(w.X, w.A, w.Qv, w.QA, 30, prec=O.F32)
    with _index(nhq, w) as ix:
        ids, g, chi = empty_out(w.nq, 30)
        nhq.nhq_brute_force(ix.handle, dev(w.Qv), dev(w.QA), 30, ids, g, chi)
        torch.cuda.synchronize()
    got = ids_i64(ids)
    assert (got == ref_ids).all()
    assert (got[:, 20:] == -1).all() and np.isinf(g.cpu().numpy()[:, 20:]).all()
    assert (chi.cpu().numpy()[:, 20:] == 255).all()


# ------------------------------------------------------------------ candidates (Sec. 4.1)
@pytest.mark.parametrize("weights", [None, CONST])
def test_knn_exact_on_integer_data(nhq, weights):
    w = synth.int_valued(2500, 1, 32, seed=36)
    ref, _ = O.knn(w.X, w.A, 64, weights=weights, prec=O.F32)
    with _index(nhq, w, weights) as ix:
        cand = torch.empty((w.N, 64), dtype=torch.uint32, device="cuda:0")
        nhq.nhq_knn(ix.handle, 64, cand)
        torch.cuda.synchronize()
    assert (ids_i64(cand) == ref).all()


# ------------------------------------------------------------------ edge selection (Def. 6)
@pytest.mark.parametrize("weights", [None, CONST])
@pytest.mark.parametrize("R", [8, 32])
def test_edge_select_exact_on_integer_data(nhq, weights, R):
    w = synth.int_valued(2000, 1, 24, seed=37)
    cand, _ = O.knn(w.X, w.A, 48, weights=weights, prec=O.F32)
    ref, deg = O.edge_select(w.X, w.A, cand, R, weights=weights, prec=O.F32)
    with _index(nhq, w, weights) as ix:
        out = torch.empty((w.N, R), dtype=torch.uint32, device="cuda:0")
        nhq.nhq_edge_select(ix.handle, dev(to_u32_graph(cand)), R, out)
        torch.cuda.synchronize()
    assert (ids_i64(out) == ref).all()


def test_edge_select_skips_self_repeats_and_padding(nhq):
    w = synth.int_valued(300, 1, 8, seed=38)
    cand, _ = O.knn(w.X, w.A, 20, prec=O.F32)
    cand = cand.copy()
    cand[:, 3] = np.arange(300)          # self
    cand[:, 5] = cand[:, 0]              # repeat
    cand[:, 7] = -1                      # padding
    cand[::2, 10:] = -1                  # short rows
    ref, _ = O.edge_select(w.X, w.A, cand, 12, prec=O.F32)
    with _index(nhq, w) as ix:
        out = torch.empty((w.N, 12), dtype=torch.uint32, device="cuda:0")
        nhq.nhq_edge_select(ix.handle, dev(to_u32_graph(cand)), 12, out)
        torch.cuda.synchronize()
    assert (ids_i64(out) == ref).all()


def test_reverse_candidates_exact(nhq):
    w = synth.int_valued(1500, 1, 16, seed=39)
    cand, _ = O.knn(w.X, w.A, 32, prec=O.F32)
    nbr, _ = O.edge_select(w.X, w.A, cand, 16, prec=O.F32)
    for cap in (0, 5, 64):
        ref = O.reverse_candidates(nbr, cap=cap)
        with _index(nhq, w) as ix:
            out = torch.empty((w.N, 16 + cap), dtype=torch.uint32, device="cuda:0")
            nhq.nhq_reverse_candidates(ix.handle, dev(to_u32_graph(nbr)), cap, out)
            torch.cuda.synchronize()
        assert (ids_i64(out) == ref).all(), cap


@pytest.mark.parametrize("weights", [None, CONST])
def test_full_build_matches_oracle_build(nhq, weights):
    w = synth.int_valued(2200, 1, 32, seed=40)
    ref, _, _ = O.build_graph(w.X, w.A, R=24, K=48, weights=weights)
    with nhq.Index.build(dev(w.X), dev(w.A), degree=24, weights=weights, K=48) as ix:
        assert ix.info == (w.N, w.d, w.m, 24)
        out = torch.empty((w.N, 24), dtype=torch.uint32, device="cuda:0")
        nhq.nhq_index_get_graph(ix.handle, out)
        torch.cuda.synchronize()
    assert (ids_i64(out) == ref).all()


# ------------------------------------------------------------------ search (Alg. 2)
@pytest.fixture(scope="module")
def graph_case():
    w = synth.int_valued(4000, 96, 32, cards=(3, 5, 7), n_comp=20, seed=41)
    graphs = {}
    for name, wts in (("prop", None), ("const", CONST)):
        nbr, _, _ = O.build_graph(w.X, w.A, R=16, K=32, weights=wts)
        graphs[name] = (wts, nbr)
    return w, graphs


@pytest.mark.parametrize("wname", ["prop", "const"])
@pytest.mark.parametrize("h", [1, 2, 4])
@pytest.mark.parametrize("k,ef", [(1, 10), (10, 10), (10, 37), (10, 100)])
def test_search_exact_vs_serial_oracle(nhq, graph_case, wname, h, k, ef):
    w, graphs = graph_case
    wts, nbr = graphs[wname]
    ref = O.search(w.X, w.A, nbr, w.Qv, w.QA, k, ef, h=h, seed=77, weights=wts)
    with _index(nhq, w, wts) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, k)
        status = torch.empty(w.nq, dtype=torch.int32, device="cuda:0")
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), k, ef, ids, g, chi, status, h=h, seed=77)
        torch.cuda.synchronize()
    assert (ids_i64(ids) == ref["ids"]).all()
    assert (chi.cpu().numpy().astype(np.int32) == ref["chi"]).all()
    assert np.array_equal(g.cpu().numpy().astype(np.float64), ref["gamma"])
    assert (status.cpu().numpy() == ref["status"]).all()


def test_search_small_visited_filter_is_still_exact(nhq, graph_case):
    # a minimal filter forces repeated rebuilds; results must not change
    w, graphs = graph_case
    wts, nbr = graphs["prop"]
    ref = O.search(w.X, w.A, nbr, w.Qv, w.QA, 10, 200, seed=3, weights=wts)
    with _index(nhq, w, wts) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, 10)
        ndc = torch.empty(w.nq, dtype=torch.int32, device="cuda:0")
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 200, ids, g, chi, ndc=ndc, seed=3,
                       hash_bits=10)
        torch.cuda.synchronize()
    assert (ids_i64(ids) == ref["ids"]).all()
    assert (ndc.cpu().numpy() >= 1).all()


def test_search_iteration_cap(nhq, graph_case):
    w, graphs = graph_case
    wts, nbr = graphs["prop"]
    ref = O.search(w.X, w.A, nbr, w.Qv, w.QA, 5, 40, seed=9, max_iters=3, weights=wts)
    assert (ref["status"] == O.ITER_LIMIT).all()
    with _index(nhq, w, wts) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, 5)
        status = torch.empty(w.nq, dtype=torch.int32, device="cuda:0")
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 5, 40, ids, g, chi, status, seed=9,
                       max_iters=3)
        torch.cuda.synchronize()
    assert (status.cpu().numpy() == nhq.ERR_ITER_LIMIT).all()
    assert (ids_i64(ids) == ref["ids"]).all()


def test_search_host_pointers_match_device(nhq, graph_case):
    w, graphs = graph_case
    wts, nbr = graphs["const"]
    ref = O.search(w.X, w.A, nbr, w.Qv, w.QA, 10, 64, seed=1, weights=wts)
    with nhq.Index.create(w.X, w.A, wts) as ix:  # host vectors too
        nhq.nhq_index_set_graph(ix.handle, to_u32_graph(nbr))
        ids = np.empty((w.nq, 10), np.uint32)
        g = np.empty((w.nq, 10), np.float32)
        chi = np.empty((w.nq, 10), np.uint8)
        nhq.nhq_search(ix.handle, w.Qv, w.QA, 10, 64, ids, g, chi, seed=1)
    assert (ids_i64(ids) == ref["ids"]).all()
    assert np.array_equal(g.astype(np.float64), ref["gamma"])


def test_search_batched_mixed_k_ef(nhq, graph_case):
    w, graphs = graph_case
    wts, nbr = graphs["const"]
    k_arr, ef_arr = synth.mixed_k_ef(w.nq, seed=5, ks=(1, 10, 20), ef_lo=16, ef_hi=120)
    k_max = int(k_arr.max())
    with _index(nhq, w, wts) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, k_max)
        nhq.nhq_search_batched(ix.handle, dev(w.Qv), dev(w.QA), dev(k_arr), dev(ef_arr), k_max,
                               ids, g, chi, seed=4)
        torch.cuda.synchronize()
    got = ids_i64(ids)
    # the oracle numbers queries by their row in its call, so run it on the whole
    # batch once per distinct (k, ef) and compare the rows that use that pair
    for kk, ee in sorted(set(zip(k_arr.tolist(), ef_arr.tolist()))):
        r = O.search(w.X, w.A, nbr, w.Qv, w.QA, kk, ee, seed=4, weights=wts)
        rows = np.nonzero((k_arr == kk) & (ef_arr == ee))[0]
        assert (got[rows, :kk] == r["ids"][rows]).all(), (kk, ee)
        assert (got[rows, kk:] == -1).all()


def test_search_bf16_scoring_exact_on_small_integers(nhq, graph_case):
    # integer components 0..255 are exact in bf16, so bf16 scoring changes nothing
    w, graphs = graph_case
    wts, nbr = graphs["prop"]
    ref = O.search(w.X, w.A, nbr, w.Qv, w.QA, 10, 50, seed=8, weights=wts)
    with _index(nhq, w, wts) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 50, ids, g, chi, seed=8,
                       vec_dtype=nhq.VEC_BF16)
        torch.cuda.synchronize()
    assert (ids_i64(ids) == ref["ids"]).all()


# ------------------------------------------------------------------ edge cases
def test_search_tiny_graph_degree_64_and_gaps(nhq):
    # N below the seed count, degree 64 (two slots per lane), sentinels inside rows
    w = synth.int_valued(90, 20, 3, cards=(2,), seed=42)
    r = np.random.default_rng(0)
    nbr = np.array([r.permutation([j for j in range(90) if j != i])[:64] for i in range(90)])
    nbr[r.random(nbr.shape) < 0.2] = -1
    for ef in (10, 90):
        ref = O.search(w.X, w.A, nbr, w.Qv, w.QA, 10, ef, h=2, seed=6)
        with _index(nhq, w) as ix:
            nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
            ids, g, chi = empty_out(w.nq, 10)
            nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, ef, ids, g, chi, h=2, seed=6)
            torch.cuda.synchronize()
        assert (ids_i64(ids) == ref["ids"]).all(), ef


def test_search_ef_equal_N_reaches_brute_force_on_connected_graph(nhq):
    w = synth.int_valued(700, 30, 12, seed=43)
    nbr, _, _ = O.build_graph(w.X, w.A, R=12, K=24)
    ref_bf, _, _ = O.fused_topk(w.X, w.A, w.Qv, w.QA, 10, prec=O.F32)
    with _index(nhq, w) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 700, ids, g, chi, seed=2)
        torch.cuda.synchronize()
    ref = O.search(w.X, w.A, nbr, w.Qv, w.QA, 10, 700, seed=2)
    assert (ids_i64(ids) == ref["ids"]).all()
    # with every vertex reachable the exhaustive search is the brute-force answer
    assert (ids_i64(ids) == ref_bf).mean() > 0.99


@pytest.mark.parametrize("d,m", [(1, 1), (3, 4), (130, 2)])
def test_odd_dimensions_and_attribute_counts(nhq, d, m):
    cards = (4, 3, 2, 5)[:m]
    w = synth.int_valued(600, 17, d, cards=cards, seed=44 + d)
    ref_ids, _, ref_chi = O.fused_topk(w.X, w.A, w.Qv, w.QA, 7, prec=O.F32)
    nbr, _, _ = O.build_graph(w.X, w.A, R=8, K=16)
    sref = O.search(w.X, w.A, nbr, w.Qv, w.QA, 7, 20, seed=1)
    with _index(nhq, w) as ix:
        ids, g, chi = empty_out(w.nq, 7)
        nhq.nhq_brute_force(ix.handle, dev(w.Qv), dev(w.QA), 7, ids, g, chi)
        torch.cuda.synchronize()
        assert (ids_i64(ids) == ref_ids).all()
        assert (chi.cpu().numpy() == ref_chi).all()
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 7, 20, ids, g, chi, seed=1)
        torch.cuda.synchronize()
        assert (ids_i64(ids) == sref["ids"]).all()


def test_empty_batch_and_argument_errors(nhq, graph_case):
    w, graphs = graph_case
    with _index(nhq, w) as ix:
        e = torch.empty((0, 10), dtype=torch.uint32, device="cuda:0")
        with pytest.raises(nhq.NHQError):  # no graph yet
            nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 10, empty_out(w.nq, 10)[0])
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(graphs["prop"][1])))
        nhq.nhq_search(ix.handle, dev(w.Qv[:0]), dev(w.QA[:0]), 10, 10, e)  # Q = 0: no-op
        with pytest.raises(nhq.NHQError):  # ef < k
            nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 5, empty_out(w.nq, 10)[0])
        bad = to_u32_graph(graphs["prop"][1]).copy()
        bad[5, 0] = w.N + 3
        with pytest.raises(nhq.NHQError):  # out-of-range neighbour id
            nhq.nhq_index_set_graph(ix.handle, dev(bad))
    with pytest.raises(nhq.NHQError):  # non-finite vector
        X = w.X.copy()
        X[3, 2] = np.nan
        nhq.Index.create(dev(X), dev(w.A))


def test_save_load_roundtrip(nhq, graph_case, tmp_path):
    w, graphs = graph_case
    wts, nbr = graphs["const"]
    p = str(tmp_path / "ix.nhq")
    with _index(nhq, w, wts) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        nhq.nhq_save(ix.handle, p)
        a = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 40, *a, seed=3)
    with nhq.Index(nhq.nhq_load(p)) as ix2:
        assert ix2.info == (w.N, w.d, w.m, 16)
        b = empty_out(w.nq, 10)
        nhq.nhq_search(ix2.handle, dev(w.Qv), dev(w.QA), 10, 40, *b, seed=3)
        torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


# ------------------------------------------------------------------ seed sets B
@pytest.mark.parametrize("wname", ["prop", "const"])
@pytest.mark.parametrize("ef", [10, 20, 64])
def test_search_attribute_entry_seeds_exact(nhq, graph_case, wname, ef):
    w, graphs = graph_case
    wts, nbr = graphs[wname]
    QA = w.QA.copy()
    QA[::7, 0] = 200  # tuples that no object has: the random stream is used for them
    ref = O.search(w.X, w.A, nbr, w.Qv, QA, 10, ef, seed=21, weights=wts,
                   seed_mode=O.SEED_ATTRIBUTE)
    with _index(nhq, w, wts) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, 10)
        ndc = torch.empty(w.nq, dtype=torch.int32, device="cuda:0")
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(QA), 10, ef, ids, g, chi, ndc=ndc, seed=21,
                       seed_mode=nhq.SEED_ATTRIBUTE)
        torch.cuda.synchronize()
    assert (ids_i64(ids) == ref["ids"]).all()
    assert np.array_equal(g.cpu().numpy().astype(np.float64), ref["gamma"])


@pytest.mark.parametrize("cards,ef,d", [((3, 5, 7), 10, 40), ((3, 5, 7), 64, 40),
                                        ((2,), 10, 40), ((2,), 64, 40), ((2,), 64, 30)])
def test_search_nearest_attribute_entry_seeds_exact(nhq, cards, ef, d):
    # (3, 5, 7): every run is shorter than 256, so all members are ranked; (2,): runs of
    # about 2000, so 256 evenly spaced members are sampled and ranked; d = 30 takes the
    # scalar row loop, d = 40 the 4-wide one
    w = synth.int_valued(3000, 64, d, cards=cards, n_comp=12, seed=43)
    nbr, _, _ = O.build_graph(w.X, w.A, R=16, K=32, weights=CONST)
    QA = w.QA.copy()
    QA[::9, 0] = 200  # tuples that no object has: the random stream is used for them
    ref = O.search(w.X, w.A, nbr, w.Qv, QA, 10, ef, seed=23, weights=CONST,
                   seed_mode=O.SEED_ATTRIBUTE_NEAR)
    with _index(nhq, w, CONST) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(QA), 10, ef, ids, g, chi, seed=23,
                       seed_mode=nhq.SEED_ATTRIBUTE_NEAR)
        torch.cuda.synchronize()
    assert (ids_i64(ids) == ref["ids"]).all()
    assert (chi.cpu().numpy().astype(np.int32) == ref["chi"]).all()
    assert np.array_equal(g.cpu().numpy().astype(np.float64), ref["gamma"])


def test_search_given_seeds_exact(nhq, graph_case):
    w, graphs = graph_case
    wts, nbr = graphs["const"]
    r = np.random.default_rng(3)
    seeds = r.integers(0, w.N, (w.nq, 64)).astype(np.int64)
    seeds[:, 5] = seeds[:, 0]           # repeats
    seeds[r.random(seeds.shape) < 0.3] = -1
    ref = O.search(w.X, w.A, nbr, w.Qv, w.QA, 10, 40, weights=wts, seeds=seeds)
    with _index(nhq, w, wts) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 40, ids, g, chi,
                       seeds=dev(to_u32_graph(seeds)))
        torch.cuda.synchronize()
        # host seed array through the same call
        ids2, g2, chi2 = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 40, ids2, g2, chi2,
                       seeds=to_u32_graph(seeds))
        torch.cuda.synchronize()
    assert (ids_i64(ids) == ref["ids"]).all()
    assert torch.equal(ids, ids2)


# ------------------------------------------------------------------ reduced-precision scoring
@pytest.mark.parametrize("vec,rnd", [(1, 1), (2, 2), (3, 3)])
@pytest.mark.parametrize("rerank", [False, True])
def test_search_reduced_precision_exact_on_integer_data(nhq, graph_case, vec, rnd, rerank):
    # 0..255 components round to integers in bf16, fp8 e4m3 and f16, so the scoring
    # distances stay exact in f32 and the search must equal the oracle's bit for bit
    w, graphs = graph_case
    wts, nbr = graphs["const"]
    ref = O.search(w.X, w.A, nbr, w.Qv, w.QA, 10, 40, seed=5, weights=wts, vec_round=rnd,
                   rerank=rerank, seed_mode=O.SEED_ATTRIBUTE)
    with _index(nhq, w, wts) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 40, ids, g, chi, seed=5,
                       vec_dtype=vec, rerank=int(rerank), seed_mode=nhq.SEED_ATTRIBUTE)
        torch.cuda.synchronize()
    assert (ids_i64(ids) == ref["ids"]).all()
    assert np.array_equal(g.cpu().numpy().astype(np.float64), ref["gamma"])
    assert (chi.cpu().numpy().astype(np.int32) == ref["chi"]).all()


def test_search_rerank_on_float_data(nhq):
    # unit-normalised float rows: bf16 / fp8 scoring with an f32 re-rank; values must
    # be the exact f32 Gamma of the returned ids and ids equal up to near-ties
    w = synth.c3(N=3000, nq=40, d=96, cards=(2, 5), n_comp=20, seed=45)
    nbr, _, _ = O.build_graph(w.X, w.A, R=16, K=32, prec=O.F32)
    for vec, rnd in ((1, O.ROUND_BF16), (2, O.ROUND_E4M3), (3, O.ROUND_F16)):
        ref = O.search(w.X, w.A, nbr, w.Qv, w.QA, 10, 48, seed=2, vec_round=rnd, rerank=True)
        with _index(nhq, w) as ix:
            nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
            ids, g, chi = empty_out(w.nq, 10)
            nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 48, ids, g, chi, seed=2,
                           vec_dtype=vec, rerank=1)
            torch.cuda.synchronize()
        got, gg = ids_i64(ids), g.cpu().numpy()
        for q in range(w.nq):
            exact = [O.gamma(O.delta(w.Qv[q], w.X[i], O.F64), O.chi(w.QA[q], w.A[i]), w.m)
                     for i in got[q]]
            assert np.allclose(gg[q], exact, rtol=1e-5, atol=0)
            assert (np.diff(gg[q]) >= 0).all()
        # the pool decisions use the rounded copy; ids may differ only where the
        # rounded Gammas nearly tie, so require a high overlap with the oracle
        overlap = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(got, ref["ids"])])
        assert overlap > 0.97, (vec, overlap)


# ------------------------------------------------------------------ tensor-core candidates
@pytest.mark.parametrize("weights", [None, CONST])
@pytest.mark.parametrize("N,d", [(2500, 32), (2500, 128), (300, 64), (1500, 200)])
def test_knn_tensor_cores_exact_on_integer_data(nhq, weights, N, d):
    w = synth.int_valued(N, 1, d, seed=60 + d)
    ref, ref_g = O.knn(w.X, w.A, 64, weights=weights, prec=O.F32)
    with _index(nhq, w, weights) as ix:
        cand = torch.empty((w.N, 64), dtype=torch.uint32, device="cuda:0")
        dist = torch.empty((w.N, 64), dtype=torch.float32, device="cuda:0")
        nhq.nhq_knn_bf16(ix.handle, 64, cand, dist)
        torch.cuda.synchronize()
    assert (ids_i64(cand) == ref).all()
    assert np.array_equal(dist.cpu().numpy().astype(np.float64), ref_g)


@pytest.mark.parametrize("weights", [None, CONST])
def test_knn_tensor_cores_exact_with_long_tuple_runs(nhq, weights):
    # six attribute tuples: most column tiles hold a single tuple (the per-tile chi
    # path), and rows whose lists are full of matching objects reject whole tiles
    w = synth.int_valued(3001, 1, 48, cards=(2, 3), n_comp=12, seed=63)
    ref, ref_g = O.knn(w.X, w.A, 24, weights=weights, prec=O.F32)
    with _index(nhq, w, weights) as ix:
        cand = torch.empty((w.N, 24), dtype=torch.uint32, device="cuda:0")
        dist = torch.empty((w.N, 24), dtype=torch.float32, device="cuda:0")
        nhq.nhq_knn_bf16(ix.handle, 24, cand, dist)
        torch.cuda.synchronize()
    assert (ids_i64(cand) == ref).all()
    assert np.array_equal(dist.cpu().numpy().astype(np.float64), ref_g)


@pytest.mark.parametrize("weights", [None, CONST])
@pytest.mark.parametrize("d", [96, 960])
def test_knn_tensor_cores_on_float_data(nhq, weights, d):
    # Float rows: the kernel rounds every row to bf16 and forms delta^2 as
    # |u|^2 + |v|^2 - 2 u.v in f32, so its candidate sets are the K nearest of the rounded
    # rows up to that formula's rounding.  Against the oracle's canonical-f32 sets of the
    # rounded rows (ties in f32 Gamma broken by id on both sides), on sampled vertices:
    # every Gamma within 1e-5 relative, ids equal except at near-ties, where the two f64
    # Gammas differ by less than the delta error (1e-5 delta, times w_v) plus two ulps of
    # the f32 Gamma, and such swaps are rare.  d = 96 is the c4/c5 row shape (mixture,
    # sigma 0.3); d = 960 the c3 shape (unit rows).
    N, K = 20000, 64
    if d == 96:
        w = synth.c4(N=N, nq=1, d=96, n_comp=200, seed=68)
    else:
        w = synth.c3(N=N, nq=1, d=960, n_comp=200, seed=69)
    rows = np.random.default_rng(70).choice(N, 150, replace=False)
    ref, ref_g = O.knn(w.X, w.A, K, weights=weights, prec=O.F32, rows=rows,
                       vec_round=O.ROUND_BF16)
    with _index(nhq, w, weights) as ix:
        cand = torch.empty((w.N, K), dtype=torch.uint32, device="cuda:0")
        dist = torch.empty((w.N, K), dtype=torch.float32, device="cuda:0")
        nhq.nhq_knn_bf16(ix.handle, K, cand, dist)
        torch.cuda.synchronize()
    got, gg = ids_i64(cand)[rows], dist.cpu().numpy()[rows]
    assert not (ids_i64(cand) == np.arange(N)[:, None]).any()
    Xr = O.round_rows(w.X, O.ROUND_BF16).astype(np.float64)
    wv = 1.0 if weights is None else weights[0]

    def f64(u, ids):  # f64 Gamma and delta of the rounded rows
        dl = np.sqrt(((Xr[ids] - Xr[u]) ** 2).sum(-1))
        ch = (w.A[ids] != w.A[u]).sum(-1)
        g = dl * (1 + ch / w.m) if weights is None else weights[0] * dl + weights[1] * ch
        return g, dl

    swaps = 0
    for r, u in enumerate(rows):
        assert np.allclose(gg[r], ref_g[r], rtol=1e-5, atol=0), r
        assert (np.diff(gg[r].astype(np.float64)) >= 0).all()
        if (got[r] == ref[r]).all():
            continue
        ga, da = f64(u, got[r])
        gb, db = f64(u, ref[r])
        tol = 1e-5 * wv * np.maximum(da, db) + 2 * np.spacing(gg[r]).astype(np.float64)
        assert (np.abs(ga - gb) <= tol).all(), r
        assert len(set(got[r].tolist())) == K
        swaps += int((got[r] != ref[r]).sum())
    assert swaps <= 0.01 * got.size, swaps


def test_build_with_tensor_core_candidates_equals_f32_build(nhq):
    w = synth.int_valued(2200, 1, 32, seed=62)
    ref, _, _ = O.build_graph(w.X, w.A, R=24, K=48, weights=CONST)
    with nhq.Index.build(dev(w.X), dev(w.A), degree=24, weights=CONST, K=48, knn_dtype=1) as ix:
        out = torch.empty((w.N, 24), dtype=torch.uint32, device="cuda:0")
        nhq.nhq_index_get_graph(ix.handle, out)
        torch.cuda.synchronize()
    assert (ids_i64(out) == ref).all()
