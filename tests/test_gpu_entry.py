"""Entry cells and the learned entry model (a project addition): the cell assignment,
the nearest-cell and learned seed rules, the model's forward pass, gradient and
training, all through the C ABI against the oracle (oracle.cells / nearest_cells /
cell_seeds, oracle/mlp.py)."""
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


@pytest.fixture(scope="module")
def case():
    w = synth.int_valued(4000, 300, 24, cards=(2, 3, 3), n_comp=30, seed=81)
    nbr, _, _ = O.build_graph(w.X, w.A, R=16, K=32, weights=CONST)
    return w, nbr


def _model(d, E, seed, scale=0.02):
    rng = np.random.default_rng(seed)
    p = (rng.standard_normal(mlp.entry_size(d, E)) * 0.2).astype(np.float32)
    p[0] = scale
    return p


def test_cells_are_the_nearest_centroids(nhq, case):
    w, _ = case
    with nhq.Index.create(dev(w.X), dev(w.A), CONST) as ix:
        for E in (1, 37, 200):
            nhq.nhq_index_build_cells(ix.handle, E)
            cell = torch.empty(w.N, dtype=torch.uint32, device="cuda:0")
            assert nhq.nhq_index_cells(ix.handle, cell) == E
            torch.cuda.synchronize()
            assert (cell.cpu().numpy().astype(np.int64) == O.cells(w.X, E)).all(), E
        with pytest.raises(nhq.NHQError):
            nhq.nhq_index_build_cells(ix.handle, 0)


def test_entry_forward_matches_the_oracle(nhq):
    d, E, n = 40, 70, 300
    p = _model(d, E, 82)
    Q = np.random.default_rng(83).standard_normal((n, d)).astype(np.float32) * 30
    logits = torch.empty((n, E), dtype=torch.float32, device="cuda:0")
    nhq.nhq_entry_forward(dev(p), E, dev(Q), logits)
    torch.cuda.synchronize()
    # the search reads fp16 weights; the input scale stays f32
    p16 = mlp.round_f16(p)
    p16[0] = p[0]
    want = mlp.entry_forward(p16, Q, d, E)
    assert np.allclose(logits.cpu().numpy(), want, rtol=1e-4, atol=1e-4)


def test_entry_gradient_matches_the_oracle(nhq):
    d, E, n = 24, 33, 5000  # several chunks of the gradient pass
    p = _model(d, E, 84)
    rng = np.random.default_rng(85)
    Q = rng.standard_normal((n, d)).astype(np.float32) * 20
    y = rng.integers(0, E, n).astype(np.int32)
    y[::97] = -1  # ignored samples
    grad = torch.empty(p.size, dtype=torch.float32, device="cuda:0")
    loss = torch.empty(1, dtype=torch.float32, device="cuda:0")
    nhq.nhq_entry_grad(dev(p), E, dev(Q), dev(y), grad, loss)
    torch.cuda.synchronize()
    keep = y >= 0
    lw, gw = mlp.entry_loss_and_grad(p.astype(np.float64), Q[keep], y[keep], d, E)
    # the library divides by all n samples; the ignored ones contribute nothing
    frac = keep.sum() / n
    g = grad.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - lw * frac) < 1e-4 * abs(lw)
    assert g[0] == 0.0
    assert np.allclose(g, gw * frac, rtol=1e-3, atol=1e-6 * np.abs(gw).max())


def test_entry_training_learns_the_cells(nhq, case):
    # labels = each training query's nearest cell: the trained model must rank it first
    # far more often than chance and lower the loss
    w, _ = case
    E = 16
    tr = synth.int_valued(4000, 6000, 24, cards=(2, 3, 3), n_comp=30, seed=81)
    y = O.nearest_cells(w.X, E, tr.Qv, 1)[:, 0].astype(np.int32)
    p = _model(24, E, 86, scale=1.0 / 64.0) * np.float32(0.1)
    p[0] = 1.0 / 64.0
    P = dev(p)
    grad = torch.empty(p.size, dtype=torch.float32, device="cuda:0")
    loss0 = torch.empty(1, dtype=torch.float32, device="cuda:0")
    Qd, yd = dev(tr.Qv), dev(y)
    nhq.nhq_entry_grad(P, E, Qd, yd, grad, loss0)
    nhq.nhq_entry_train(P, E, Qd, yd, epochs=30, batch=256, lr=3e-3)
    loss1 = torch.empty(1, dtype=torch.float32, device="cuda:0")
    nhq.nhq_entry_grad(P, E, Qd, yd, grad, loss1)
    logits = torch.empty((tr.nq, E), dtype=torch.float32, device="cuda:0")
    nhq.nhq_entry_forward(P, E, Qd, logits)
    torch.cuda.synchronize()
    acc = float((logits.argmax(1).cpu().numpy() == y).mean())
    assert loss1.item() < 0.5 * loss0.item(), (loss0.item(), loss1.item())
    assert acc > 0.8, acc
    assert P[0].item() == np.float32(1.0 / 64.0)  # the scale is not trained


def _chosen_from_logits(L, T):
    # largest logit first, ties to the smaller cell
    return np.array([np.lexsort((np.arange(L.shape[1]), -row))[:T] for row in L])


@pytest.mark.parametrize("mode", ["nearest", "learned"])
@pytest.mark.parametrize("ef,T", [(16, 1), (40, 3)])
def test_cell_seed_modes_match_the_oracle(nhq, case, mode, ef, T):
    w, nbr = case
    E = 24
    QA = w.QA.copy()
    QA[::17, 0] = 9  # no object has code 9: the random fallback
    p = _model(w.d, E, 87, scale=0.01)
    with nhq.Index.create(dev(w.X), dev(w.A), CONST) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        nhq.nhq_index_build_cells(ix.handle, E)
        ids, g, c = empty_out(w.nq, 10)
        cells = torch.empty((w.nq, T), dtype=torch.int32, device="cuda:0")
        ndc = torch.empty(w.nq, dtype=torch.int32, device="cuda:0")
        sm = nhq.SEED_CELL_NEAREST if mode == "nearest" else nhq.SEED_CELL_LEARNED
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(QA), 10, ef, ids, g, c, ndc=ndc, seed=5,
                       seed_mode=sm, entry_cells=T, cells_out=cells,
                       entry_model=dev(p) if mode == "learned" else None)
        if mode == "learned":
            logits = torch.empty((w.nq, E), dtype=torch.float32, device="cuda:0")
            nhq.nhq_entry_forward(dev(p), E, dev(w.Qv), logits)
        torch.cuda.synchronize()
    chosen = cells.cpu().numpy()
    if mode == "nearest":
        assert (chosen == O.nearest_cells(w.X, E, w.Qv, T)).all()
    else:  # the seed pass and nhq_entry_forward share their arithmetic
        assert (chosen == _chosen_from_logits(logits.cpu().numpy(), T)).all()
    B = O.cell_seeds(w.A, QA, O.cells(w.X, E), chosen, ef, seed=5)
    r = O.search(w.X, w.A, nbr, w.Qv, QA, 10, ef, weights=CONST, seeds=B, prec=O.F32)
    assert (ids_i64(ids) == r["ids"]).all()
    assert np.array_equal(g.cpu().numpy().astype(np.float64), r["gamma"])
    # under constant weights the kernel skips the distance of a neighbour whose attribute
    # term alone exceeds the pool's last record (it could not enter), which the oracle
    # evaluates: the kernel's count of distance evaluations is at most the oracle's
    assert (ndc.cpu().numpy() <= r["ndc"]).all()


def test_cell_seed_modes_refuse_bad_settings(nhq, case):
    w, nbr = case
    with nhq.Index.create(dev(w.X), dev(w.A), CONST) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        ids, g, c = empty_out(w.nq, 10)
        with pytest.raises(nhq.NHQError):  # no cells yet
            nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 20, ids, g, c,
                           seed_mode=nhq.SEED_CELL_NEAREST)
        nhq.nhq_index_build_cells(ix.handle, 4)
        for kw in (dict(entry_cells=5), dict(entry_cells=9), dict(wildcard=1)):
            with pytest.raises(nhq.NHQError):
                nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 20, ids, g, c,
                               seed_mode=nhq.SEED_CELL_NEAREST, **kw)
        with pytest.raises(nhq.NHQError):  # learned mode without a model
            nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 20, ids, g, c,
                           seed_mode=nhq.SEED_CELL_LEARNED)


def test_entry_labels_are_the_cells_of_the_first_results(nhq, case):
    w, nbr = case
    E = 12
    with nhq.Index.create(dev(w.X), dev(w.A), CONST) as ix:
        nhq.nhq_index_set_graph(ix.handle, dev(to_u32_graph(nbr)))
        nhq.nhq_index_build_cells(ix.handle, E)
        ids, g, c = empty_out(w.nq, 10)
        nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 20, ids, g, c,
                       seed_mode=nhq.SEED_ATTRIBUTE)
        ids[5, 0] = 0xFFFFFFFF
        lab = torch.empty(w.nq, dtype=torch.int32, device="cuda:0")
        nhq.nhq_entry_labels(ix.handle, ids, lab)
        torch.cuda.synchronize()
    cell_of = O.cells(w.X, E)
    first = ids_i64(ids)[:, 0]
    want = np.where(first >= 0, cell_of[np.maximum(first, 0)], -1)
    assert (lab.cpu().numpy() == want).all()
