"""The learned early stop: MLP kernels against the fp64 oracle, the exact
limits of the learned search, the trace labels, and what the trained model
gains over the plain search."""
import numpy as np
import pytest

import oracle as O
import synth
from helpers import dev, empty_out, ids_i64, to_u32_graph
from oracle import mlp

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


def _params(seed, scale=0.3, b2=0.0):
    r = np.random.default_rng(seed)
    p = (r.standard_normal(mlp.N_PARAMS) * scale).astype(np.float32)
    p[-1] = b2
    return p


def test_mlp_forward_matches_oracle(nhq):
    p = _params(1)
    X = np.random.default_rng(2).standard_normal((1000, 8)).astype(np.float32)
    out = torch.empty(1000, dtype=torch.float32, device="cuda:0")
    nhq.nhq_mlp_forward(dev(p), dev(X), out)
    torch.cuda.synchronize()
    ref = mlp.forward(mlp.round_f16(p), X)  # the search reads fp16 weights
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-4, atol=1e-4)


def test_mlp_gradient_matches_oracle(nhq):
    p = _params(3)
    r = np.random.default_rng(4)
    X = r.standard_normal((3000, 8)).astype(np.float32)
    y = (r.random(3000) < 0.3).astype(np.float32)
    g = torch.empty(mlp.N_PARAMS, dtype=torch.float32, device="cuda:0")
    loss = torch.empty(1, dtype=torch.float32, device="cuda:0")
    nhq.nhq_mlp_grad(dev(p), dev(X), dev(y), g, loss)
    torch.cuda.synchronize()
    ref_loss, ref_g = mlp.loss_and_grad(p.astype(np.float64), X, y)
    assert loss.item() == pytest.approx(ref_loss, rel=1e-5)
    gg = g.cpu().numpy().astype(np.float64)
    assert np.allclose(gg, ref_g, rtol=1e-3, atol=1e-6 * np.abs(ref_g).max())


def test_mlp_training_learns_a_separable_rule(nhq):
    r = np.random.default_rng(5)
    X = r.standard_normal((20000, 8)).astype(np.float32)
    y = (X[:, 0] + 0.5 * X[:, 1] - 0.3 * X[:, 4] > 0.2).astype(np.float32)
    p = dev(_params(6, scale=0.1))
    l0, _ = mlp.loss_and_grad(p.cpu().numpy().astype(np.float64), X, y)
    nhq.nhq_mlp_train(p, dev(X), dev(y), epochs=20, batch=1024, lr=3e-3)
    torch.cuda.synchronize()
    pp = p.cpu().numpy().astype(np.float64)
    l1, _ = mlp.loss_and_grad(pp, X, y)
    acc = np.mean((mlp.forward(pp, X) > 0) == (y > 0.5))
    assert l1 < 0.5 * l0 and acc > 0.95


@pytest.fixture(scope="module")
def case(nhq):
    w = synth.int_valued(4000, 120, 32, cards=(3, 5, 7), n_comp=20, seed=41)
    nbr, _, _ = O.build_graph(w.X, w.A, R=16, K=32, weights=CONST)
    return w, nbr


def _search(nhq, w, nbr, k, ef, **kw):
    with nhq.Index.create(dev(w.X), dev(w.A), CONST) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, chi = empty_out(w.nq, k)
        ex = torch.empty(w.nq, dtype=torch.int32, device="cuda:0")
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), k, ef, ids, g, chi, expansions=ex,
                       seed_mode=nhq.SEED_ATTRIBUTE, **kw)
        torch.cuda.synchronize()
    return ids_i64(ids), g.cpu().numpy(), ex.cpu().numpy()


def test_learned_stop_limits_are_exact(nhq, case):
    w, nbr = case
    ref = O.search(w.X, w.A, nbr, w.Qv, w.QA, 10, 40, weights=CONST, seed_mode=O.SEED_ATTRIBUTE)
    never = dev(_params(7, b2=-100.0))
    ids, g, _ = _search(nhq, w, nbr, 10, 40, stop_model=never, stop_threshold=0.5, stop_min=2)
    assert (ids == ref["ids"]).all()
    always = dev(_params(8, scale=0.0, b2=100.0))
    ids, _, ex = _search(nhq, w, nbr, 10, 40, stop_model=always, stop_threshold=0.5, stop_min=3)
    cap = O.search(w.X, w.A, nbr, w.Qv, w.QA, 10, 40, weights=CONST, max_iters=3,
                   seed_mode=O.SEED_ATTRIBUTE)
    assert (ids == cap["ids"]).all() and (ex == 3).all()


def test_trace_labels_match_truncated_searches(nhq, case):
    w, nbr = case
    k, ef = 10, 40
    cap = 20000
    feats = torch.empty((cap, 8), dtype=torch.float32, device="cuda:0")
    labels = torch.empty(cap, dtype=torch.uint8, device="cuda:0")
    tq = torch.empty(cap, dtype=torch.int32, device="cuda:0")
    with nhq.Index.create(dev(w.X), dev(w.A), CONST) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        n = nhq.nhq_search_trace(ix.handle, dev(w.Qv), dev(w.QA), k, ef, feats, labels, tq,
                                 stop_min=1, stop_every=1, seed_mode=nhq.SEED_ATTRIBUTE)
        torch.cuda.synchronize()
    assert 0 < n < cap
    F, L, Tq = feats[:n].cpu().numpy(), labels[:n].cpu().numpy(), tq[:n].cpu().numpy()
    assert set(np.unique(L)) <= {0, 1} and np.isfinite(F).all()
    iters = np.rint(np.expm1(F[:, 0] * 4.0)).astype(int)   # f0 = log1p(expansions) / 4
    final = O.search(w.X, w.A, nbr, w.Qv, w.QA, k, ef, weights=CONST,
                     seed_mode=O.SEED_ATTRIBUTE)["ids"]
    checked = 0
    for c in sorted(set(iters.tolist()))[:12]:
        part = O.search(w.X, w.A, nbr, w.Qv, w.QA, k, ef, weights=CONST, max_iters=int(c),
                        seed_mode=O.SEED_ATTRIBUTE)["ids"]
        sel = np.nonzero(iters == c)[0]
        for t in sel:
            want = int((part[Tq[t]] == final[Tq[t]]).all())
            assert L[t] == want, (t, c)
            checked += 1
    assert checked > 100


def test_learned_stop_gains_over_plain_search(nhq):
    # train on traces of one query set, measure on another from the same mixture
    w = synth.int_valued(20000, 3000, 32, cards=(3, 5, 7), n_comp=40, seed=46)
    k, ef = 10, 48
    with nhq.Index.build(dev(w.X), dev(w.A), degree=24, weights=CONST, K=48) as ix:
        Qtr, QAtr = dev(w.Qv[:2000]), dev(w.QA[:2000])
        Qte, QAte = dev(w.Qv[2000:]), dev(w.QA[2000:])
        cap = 200000
        feats = torch.empty((cap, 8), dtype=torch.float32, device="cuda:0")
        labels = torch.empty(cap, dtype=torch.uint8, device="cuda:0")
        tq = torch.empty(cap, dtype=torch.int32, device="cuda:0")
        n = nhq.nhq_search_trace(ix.handle, Qtr, QAtr, k, ef, feats, labels, tq, stop_min=4,
                                 stop_every=2, seed_mode=nhq.SEED_ATTRIBUTE)
        perm = torch.randperm(n, generator=torch.Generator().manual_seed(0)).to("cuda:0")
        F = feats[:n][perm].contiguous()
        Y = labels[:n][perm].to(torch.float32).contiguous()
        p = dev(_params(9, scale=0.1, b2=0.0))
        nhq.nhq_mlp_train(p, F, Y, epochs=8, batch=2048, lr=2e-3)
        nte = 1000
        ids0, g0, c0 = empty_out(nte, k)
        ex0 = torch.empty(nte, dtype=torch.int32, device="cuda:0")
        nhq.nhq_search(ix.handle, Qte, QAte, k, ef, ids0, g0, c0, expansions=ex0,
                       seed_mode=nhq.SEED_ATTRIBUTE)
        ids1, g1, c1 = empty_out(nte, k)
        ex1 = torch.empty(nte, dtype=torch.int32, device="cuda:0")
        nhq.nhq_search(ix.handle, Qte, QAte, k, ef, ids1, g1, c1, expansions=ex1,
                       seed_mode=nhq.SEED_ATTRIBUTE, stop_model=p, stop_threshold=0.95,
                       stop_min=4, stop_every=2)
        gt = torch.empty((nte, k), dtype=torch.uint32, device="cuda:0")
        nhq.nhq_brute_force(ix.handle, Qte, QAte, k, gt, weights="filter")

        # the time of both forms on this batch (CUDA events, 20 launches each)
        def timed(**kw):
            for _ in range(3):
                nhq.nhq_search(ix.handle, Qte, QAte, k, ef, ids0, g0, c0,
                               seed_mode=nhq.SEED_ATTRIBUTE, **kw)
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record()
            for _ in range(20):
                nhq.nhq_search(ix.handle, Qte, QAte, k, ef, ids0, g0, c0,
                               seed_mode=nhq.SEED_ATTRIBUTE, **kw)
            a1.record()
            a1.synchronize()
            return a0.elapsed_time(a1) / 20

        ms_plain = timed()
        ms_learned = timed(stop_model=p, stop_threshold=0.95, stop_min=4, stop_every=2)
        torch.cuda.synchronize()
    gt_i, i0, i1 = ids_i64(gt), ids_i64(ids0), ids_i64(ids1)
    rec0 = np.mean([len(set(a) & set(b[b >= 0])) / max(1, (b >= 0).sum()) for a, b in zip(i0, gt_i)])
    rec1 = np.mean([len(set(a) & set(b[b >= 0])) / max(1, (b >= 0).sum()) for a, b in zip(i1, gt_i)])
    e0, e1 = ex0.float().mean().item(), ex1.float().mean().item()
    print(f"plain: recall {rec0:.4f}, expansions {e0:.1f}, {ms_plain:.4f} ms; learned: "
          f"recall {rec1:.4f}, expansions {e1:.1f}, {ms_learned:.4f} ms "
          f"({ms_plain / ms_learned:.2f}x)")
    assert e1 < 0.85 * e0          # at least 15% fewer expansions
    assert rec1 > rec0 - 0.01      # for at most 0.01 of recall
    # Time: the gain in expansions does not turn into a gain in time (the model costs a
    # 641-parameter evaluation every second expansion, and a batch's time follows its
    # slowest queries more than its mean expansion count; on the 1M sets the learned stop
    # is not faster at the 0.95 point).  The times are printed above; the test only
    # bounds the cost of the model, at most 1.5x the plain search.
    assert ms_learned < 1.5 * ms_plain, (ms_plain, ms_learned)
