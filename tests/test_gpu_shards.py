"""Object shards (the paper's parallel form, Sec. 6.1): the object set split into P
contiguous shards with one index each, every shard searched for every query, and the
per-shard lists merged by (Gamma, global id) with nhq_merge_topk."""
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


def _stack(P, nq, k):
    return (torch.empty((P, nq, k), dtype=torch.uint32, device="cuda:0"),
            torch.empty((P, nq, k), dtype=torch.float32, device="cuda:0"),
            torch.empty((P, nq, k), dtype=torch.uint8, device="cuda:0"))


@pytest.mark.parametrize("weights", [None, CONST])
def test_merged_brute_force_equals_the_unsharded_one(nhq, weights):
    w = synth.int_valued(5000, 64, 32, seed=70)
    cuts = [0, 1100, 2600, 2607, 5000]  # uneven, one shard smaller than k
    P, k = len(cuts) - 1, 10
    ids, d, c = _stack(P, w.nq, k)
    for p in range(P):
        lo, hi = cuts[p], cuts[p + 1]
        with nhq.Index.create(dev(w.X[lo:hi]), dev(w.A[lo:hi]), weights) as ix:
            nhq.nhq_brute_force(ix.handle, dev(w.Qv), dev(w.QA), k, ids[p], d[p], c[p])
    mi, md, mc = empty_out(w.nq, k)
    nhq.nhq_merge_topk(ids, d, dev(np.array(cuts[:P], np.uint32)), k, mi, md, chi=c, out_chi=mc)
    fi, fd, fc = empty_out(w.nq, k)
    with nhq.Index.create(dev(w.X), dev(w.A), weights) as ix:
        nhq.nhq_brute_force(ix.handle, dev(w.Qv), dev(w.QA), k, fi, fd, fc)
    torch.cuda.synchronize()
    assert torch.equal(mi, fi) and torch.equal(md, fd) and torch.equal(mc, fc)
    ref = O.fused_topk(w.X, w.A, w.Qv, w.QA, k, weights=weights, prec=O.F32)[0]
    assert (ids_i64(mi) == ref).all()


def test_merged_graph_searches_match_the_oracle(nhq):
    w = synth.int_valued(4500, 80, 32, cards=(3, 5, 7), n_comp=20, seed=71)
    cuts = [0, 1500, 2900, 4500]
    P, k, ef = 3, 10, 48
    ids, d, c = _stack(P, w.nq, k)
    per_shard = []
    for p in range(P):
        lo, hi = cuts[p], cuts[p + 1]
        with nhq.Index.build(dev(w.X[lo:hi]), dev(w.A[lo:hi]), degree=16, weights=CONST,
                             K=32) as ix:
            g = torch.empty((hi - lo, 16), dtype=torch.uint32, device="cuda:0")
            nhq.nhq_index_get_graph(ix.handle, g)
            nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), k, ef, ids[p], d[p], c[p], seed=5,
                           seed_mode=nhq.SEED_ATTRIBUTE)
            torch.cuda.synchronize()
            r = O.search(w.X[lo:hi], w.A[lo:hi], ids_i64(g), w.Qv, w.QA, k, ef, seed=5,
                         weights=CONST, seed_mode=O.SEED_ATTRIBUTE)
            per_shard.append((np.where(r["ids"] >= 0, r["ids"] + lo, -1), r["gamma"], r["chi"]))
    mi, md, mc = empty_out(w.nq, k)
    nhq.nhq_merge_topk(ids, d, np.array(cuts[:P], np.uint32), k, mi, md, chi=c, out_chi=mc)
    torch.cuda.synchronize()
    # expected: the oracle's per-shard results, ordered by (Gamma, global id)
    all_ids = np.concatenate([s[0] for s in per_shard], axis=1)
    all_g = np.concatenate([s[1] for s in per_shard], axis=1)
    all_c = np.concatenate([s[2] for s in per_shard], axis=1)
    for q in range(w.nq):
        valid = all_ids[q] >= 0
        order = np.lexsort((all_ids[q][valid], all_g[q][valid]))[:k]
        want = all_ids[q][valid][order]
        got = ids_i64(mi)[q]
        assert (got[:len(want)] == want).all() and (got[len(want):] == -1).all()
        assert np.array_equal(md.cpu().numpy()[q][:len(want)].astype(np.float64),
                              all_g[q][valid][order])
        assert (mc.cpu().numpy()[q][:len(want)] == all_c[q][valid][order]).all()


def test_merge_edge_cases(nhq):
    # one shard: the merge is the identity; more slots than records: padding
    rng = np.random.default_rng(3)
    g = np.sort(rng.random((5, 4)).astype(np.float32), axis=1)
    ids = rng.permutation(100)[:20].reshape(5, 4).astype(np.uint32)
    ids[2, 3] = 0xFFFFFFFF
    g[2, 3] = np.inf
    out_i = np.empty((5, 6), np.uint32)
    out_g = np.empty((5, 6), np.float32)
    nhq.nhq_merge_topk(ids[None], g[None], np.array([7], np.uint32), 6, out_i, out_g)  # host arrays
    for q in range(5):
        n = 3 if q == 2 else 4
        assert (out_i[q, :n] == ids[q, :n] + 7).all() and (out_g[q, :n] == g[q, :n]).all()
        assert (out_i[q, n:] == 0xFFFFFFFF).all() and np.isinf(out_g[q, n:]).all()
