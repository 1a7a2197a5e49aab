"""Parity at the full size of the headline workload: the c2-shaped set (N = 1,000,000,
d = 128, integer components, m = 3 Zipf attributes, 10,000 queries) built and searched
with the settings bench.py times (K = 64 tensor-core candidates, R = 32, reverse pass,
constant weights (1, 10,000); search k = 10, ef = 24, h = 1, attribute-entry seeds).

Integer components make every distance exact in f32, so the oracle's f32 arithmetic and
the kernels agree bit for bit: the candidate lists and the two edge-selection passes are
compared on sampled vertices (the oracle computes those one by one), and so are the
reverse candidates; the search outputs of the first 1,500 of the 10,000 queries of one
launch (the oracle's attribute-entry seeding scans all N objects per query and the seeds
depend on the query's index, so a prefix keeps the indices), and the hybrid ground
truth on sampled queries."""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import dev, empty_out, ids_i64

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CONST = (1.0, 10000.0)
R, K, CAP = 32, 64, 64


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
def big(nhq):
    """The workload, its index built step by step (as nhq_index_build does), and the
    intermediate outputs of every step."""
    w = synth.c2()
    N = w.N
    ix = nhq.Index.create(dev(w.X), dev(w.A), CONST)
    cand = torch.empty((N, K), dtype=torch.uint32, device="cuda:0")
    candg = torch.empty((N, K), dtype=torch.float32, device="cuda:0")
    nhq.nhq_knn_bf16(ix.handle, K, cand, candg)
    nbr1 = torch.empty((N, R), dtype=torch.uint32, device="cuda:0")
    nhq.nhq_edge_select(ix.handle, cand, R, nbr1)
    rc = torch.empty((N, R + CAP), dtype=torch.uint32, device="cuda:0")
    nhq.nhq_reverse_candidates(ix.handle, nbr1, CAP, rc)
    nbr2 = torch.empty((N, R), dtype=torch.uint32, device="cuda:0")
    nhq.nhq_edge_select(ix.handle, rc, R, nbr2)
    nhq.nhq_index_set_graph(ix.handle, nbr2)
    torch.cuda.synchronize()
    out = dict(w=w, ix=ix, cand=ids_i64(cand), candg=candg.cpu().numpy(), nbr1=ids_i64(nbr1),
               rc=ids_i64(rc), nbr2=ids_i64(nbr2))
    yield out
    ix.close()


def _sample(n, count, seed):
    return np.sort(np.random.default_rng(seed).choice(n, count, replace=False))


def test_candidates_on_sampled_vertices(big):
    w = big["w"]
    rows = _sample(w.N, 12, 1)
    ref, ref_g = O.knn(w.X, w.A, K, weights=CONST, prec=O.F32, rows=rows)
    assert (big["cand"][rows] == ref).all()
    assert np.array_equal(big["candg"][rows].astype(np.float64), ref_g)


def test_edge_selection_on_sampled_vertices(big):
    w = big["w"]
    rows = _sample(w.N, 200, 2)
    ref1, _ = O.edge_select(w.X, w.A, big["cand"][rows], R, weights=CONST, prec=O.F32,
                            rows=rows)
    assert (big["nbr1"][rows] == ref1).all()
    ref2, _ = O.edge_select(w.X, w.A, big["rc"][rows], R, weights=CONST, prec=O.F32, rows=rows)
    assert (big["nbr2"][rows] == ref2).all()


def test_reverse_candidates_on_sampled_vertices(big):
    # the oracle scans every source for each listed vertex: N x R steps per vertex
    rows = _sample(big["w"].N, 64, 4)
    assert (big["rc"][rows] == O.reverse_candidates(big["nbr1"], CAP, rows=rows)).all()


def test_one_call_build_equals_the_steps(nhq, big):
    w = big["w"]
    with nhq.Index.build(dev(w.X), dev(w.A), degree=R, weights=CONST, K=K, knn_dtype=1) as ix:
        g = torch.empty((w.N, R), dtype=torch.uint32, device="cuda:0")
        nhq.nhq_index_get_graph(ix.handle, g)
        torch.cuda.synchronize()
    assert (ids_i64(g) == big["nbr2"]).all()


@pytest.mark.parametrize("vec", ["f32", "bf16+rerank"])
def test_search_launch_on_a_query_prefix(nhq, big, vec):
    """The launch bench.py times (f32), and the bf16 scoring copy with the f32 re-rank."""
    w = big["w"]
    vdt = nhq.VEC_F32 if vec == "f32" else nhq.VEC_BF16
    rerank = 0 if vec == "f32" else 1
    ids, g, chi = empty_out(w.nq, 10)
    st = torch.empty(w.nq, dtype=torch.int32, device="cuda:0")
    nhq.nhq_search(big["ix"].handle, dev(w.Qv), dev(w.QA), 10, 24, ids, g, chi, st, h=1,
                   seed=12345, vec_dtype=vdt, rerank=rerank, seed_mode=nhq.SEED_ATTRIBUTE)
    torch.cuda.synchronize()
    nq = 1500
    ref = O.search(w.X, w.A, big["nbr2"], w.Qv[:nq], w.QA[:nq], 10, 24, h=1, seed=12345,
                   weights=CONST,
                   prec=O.F32, seed_mode=O.SEED_ATTRIBUTE,
                   vec_round=O.ROUND_NONE if vec == "f32" else O.ROUND_BF16,
                   rerank=bool(rerank))
    assert (st.cpu().numpy() == 0).all()
    assert (ids_i64(ids)[:nq] == ref["ids"]).all()
    assert np.array_equal(g.cpu().numpy()[:nq].astype(np.float64), ref["gamma"])
    assert (chi.cpu().numpy()[:nq] == ref["chi"]).all()


def test_hybrid_ground_truth_on_sampled_queries(nhq, big):
    w = big["w"]
    q = _sample(w.nq, 24, 3)
    ids, g, chi = empty_out(len(q), 10)
    nhq.nhq_brute_force(big["ix"].handle, dev(w.Qv[q]), dev(w.QA[q]), 10, ids, g, chi,
                        weights="filter")
    torch.cuda.synchronize()
    ref, ref_g, _ = O.filtered_topk(w.X, w.A, w.Qv[q], w.QA[q], 10, prec=O.F32)
    assert (ids_i64(ids) == ref).all()
    got_g = g.cpu().numpy().astype(np.float64)
    assert np.array_equal(got_g[ref >= 0], ref_g[ref >= 0])
