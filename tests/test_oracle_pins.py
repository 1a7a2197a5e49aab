"""Pins for the CPU oracle: each test checks the oracle against something the
paper or mathematics fixes (closed forms, published generator outputs,
hand-derived geometry, textbook routines, invariants), never against itself."""
import math
import os

import numpy as np
import pytest
import torch

import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------ generator
def test_splitmix64_published_outputs(oracle_mod):
    want = [int(r[0]) for r in _golden_rows("splitmix64_seed1234567.txt")]
    assert oracle_mod.splitmix64_stream(1234567, 5) == want


def test_mix64_zero_and_bijective_sample(oracle_mod):
    assert oracle_mod.mix64(0) == 0  # every step of the finaliser maps 0 to 0
    outs = {oracle_mod.mix64(i) for i in range(2000)}
    assert len(outs) == 2000  # a bijection has no collisions


# ------------------------------------------------------------------ Eq. 1
def test_delta_closed_forms(oracle_mod):
    O = oracle_mod
    for prec in (O.F64, O.F32):
        assert O.delta([0, 0], [3, 4], prec) == 5.0
        assert O.delta([1, 2, 3], [1, 2, 3], prec) == 0.0
        e = np.zeros(17, np.float32)
        e[9] = -2.5
        assert O.delta(np.zeros(17), e, prec) == 2.5
    # f64 against an independent textbook routine
    r = np.random.default_rng(0)
    for d in (1, 7, 128, 960):
        x, y = r.standard_normal(d).astype(np.float32), r.standard_normal(d).astype(np.float32)
        ref = float(np.linalg.norm(x.astype(np.float64) - y.astype(np.float64)))
        assert O.delta(x, y, O.F64) == pytest.approx(ref, rel=1e-14)
        assert O.delta(x, y, O.F32) == pytest.approx(ref, rel=1e-5)


def test_delta32_exact_on_integer_vectors(oracle_mod):
    # integer components 0..255 and d <= 256: the squared distance is an integer
    # below 2^24, so f32 is exact and sqrtf is the correctly rounded sqrt
    r = np.random.default_rng(1)
    for _ in range(50):
        x = r.integers(0, 256, 128).astype(np.float32)
        y = r.integers(0, 256, 128).astype(np.float32)
        s = int(((x.astype(np.int64) - y.astype(np.int64)) ** 2).sum())
        assert oracle_mod.delta(x, y, oracle_mod.F32) == float(np.sqrt(np.float32(s)))


# ------------------------------------------------------------------ Eq. 4-5
def test_chi_hand_cases(oracle_mod):
    O = oracle_mod
    assert O.chi([1, 2, 3], [1, 2, 3]) == 0
    assert O.chi([1, 2, 3], [0, 2, 3]) == 1
    assert O.chi([1, 2, 3], [1, 0, 0]) == 2
    assert O.chi([1, 2, 3], [3, 1, 2]) == 3
    assert O.chi([255, 0, 7, 9], [255, 1, 7, 8]) == 2
    assert O.chi([4], [4]) == 0


def test_chi_is_a_metric(oracle_mod):
    r = np.random.default_rng(2)
    for _ in range(300):
        a, b, c = (r.integers(0, 3, 4).astype(np.uint8) for _ in range(3))
        ab, bc, ac = oracle_mod.chi(a, b), oracle_mod.chi(b, c), oracle_mod.chi(a, c)
        assert ab == oracle_mod.chi(b, a)
        assert 0 <= ab <= 4
        assert ac <= ab + bc


# ------------------------------------------------------------------ Eq. 6 / Sec. 3.2
def test_gamma_recommended_weights_bounds(oracle_mod):
    O = oracle_mod
    for m in (1, 2, 3, 4):
        for dl in (0.0, 0.5, 1.0, 3.7, 1234.5):
            g = [O.gamma(dl, c, m) for c in range(m + 1)]
            assert g[0] == dl  # chi = 0: no change
            assert g[m] == pytest.approx(2 * dl, rel=1e-15, abs=0)  # chi = m: doubled
            assert all(dl <= x <= 2 * dl * (1 + 1e-15) for x in g)
            assert all(g[i] <= g[i + 1] for i in range(m))


def test_gamma_constant_weights_literals(oracle_mod):
    O = oracle_mod
    assert O.gamma(2.5, 2, 3, weights=(2.0, 10.0)) == 25.0
    assert O.gamma(2.5, 2, 3, weights=(2.0, 10.0), prec=O.F32) == 25.0
    assert O.gamma(7.25, 3, 3, weights=(1.0, 0.0)) == 7.25  # w_l = 0: plain delta
    assert O.gamma(7.25, 3, 3, weights=(0.0, 1.0)) == 3.0  # w_v = 0: attributes only


# ------------------------------------------------------------------ Def. 2 / Sec. 6.1
def test_fused_topk_plain_l2_matches_torch_cdist(oracle_mod):
    O = oracle_mod
    w = synth.c1(N=700, nq=25, d=32, seed=5)
    ids, g, _ = O.fused_topk(w.X, w.A, w.Qv, w.QA, 10, weights=(1.0, 0.0))
    D = torch.cdist(torch.from_numpy(w.Qv).double(), torch.from_numpy(w.X).double())
    ref = torch.topk(D, 10, largest=False)
    assert np.allclose(g, ref.values.numpy(), rtol=1e-12)
    assert (ids == ref.indices.numpy()).mean() > 0.999  # exact ties are possible only in theory


def test_fused_topk_attribute_dominant_equals_filtered(oracle_mod):
    O = oracle_mod
    w = synth.int_valued(1500, 40, 16, cards=(2, 3), seed=11)
    f_ids, f_dl, P = O.filtered_topk(w.X, w.A, w.Qv, w.QA, 10)
    # w_l larger than any delta (<= 255 * sqrt(16)) puts every match first
    ids, g, ch = O.fused_topk(w.X, w.A, w.Qv, w.QA, 10, weights=(1.0, 10000.0))
    for q in range(w.nq):
        n = min(10, P[q])
        assert (ids[q, :n] == f_ids[q, :n]).all()
        assert (ch[q, :n] == 0).all()
        assert np.allclose(g[q, :n], f_dl[q, :n], rtol=1e-15)


def test_filtered_topk_counts_and_order(oracle_mod):
    O = oracle_mod
    w = synth.c1(N=900, nq=20, d=8, cards=(2, 2), seed=3)
    ids, dl, P = O.filtered_topk(w.X, w.A, w.Qv, w.QA, 5)
    for q in range(w.nq):
        match = np.nonzero((w.A == w.QA[q]).all(axis=1))[0]
        assert P[q] == len(match)
        dd = np.linalg.norm(w.X[match].astype(np.float64) - w.Qv[q], axis=1)
        order = match[np.lexsort((match, dd))][:5]
        assert (ids[q, : len(order)] == order).all()


def test_fused_topk_hand_enumeration(oracle_mod):
    O = oracle_mod
    # 1-D points at 0..5, query at 2.2 with attribute 1; objects 1 and 4 mismatch
    X = np.arange(6, dtype=np.float32)[:, None]
    A = np.array([[1], [0], [1], [1], [0], [1]], np.uint8)
    ids, g, ch = O.fused_topk(X, A, np.array([[2.2]], np.float32), np.array([[1]], np.uint8), 6)
    # proportional weights, m = 1: Gamma = delta * (1 + chi)
    want = sorted(((abs(i - 2.2) * (1 + int(A[i, 0] != 1)), i) for i in range(6)))
    assert list(ids[0]) == [i for _, i in want]
    assert list(ch[0]) == [int(A[i, 0] != 1) for _, i in want]
    assert list(ids[0]) == [2, 3, 0, 1, 5, 4]  # Gamma: .2 .8 2.2 2.4 2.8 3.6


# ------------------------------------------------------------------ Sec. 4.1 candidates
def test_knn_excludes_self_and_matches_cdist(oracle_mod):
    O = oracle_mod
    w = synth.c1(N=400, nq=1, d=24, seed=8)
    ids, g = O.knn(w.X, w.A, 12, weights=(1.0, 0.0))
    D = torch.cdist(torch.from_numpy(w.X).double(), torch.from_numpy(w.X).double())
    D.fill_diagonal_(float("inf"))
    ref = torch.topk(D, 12, largest=False)
    assert not (ids == np.arange(400)[:, None]).any()
    assert np.allclose(g, ref.values.numpy(), rtol=1e-12)
    assert (ids == ref.indices.numpy()).mean() > 0.999


def test_graph_quality_of_exact_knn_is_one(oracle_mod):
    O = oracle_mod
    w = synth.c1(N=300, nq=1, d=16, seed=9)
    ids, _ = O.knn(w.X, w.A, 20)
    assert O.graph_quality(ids[:, :8], ids) == 1.0  # Eq. 7 with N(u) = M(u)
    r = np.random.default_rng(0)
    rnd = r.integers(0, 300, (300, 8))
    assert O.graph_quality(rnd, ids) < 0.2


# ------------------------------------------------------------------ Sec. 4.1 edge selection
def _lz_points():
    rows = _golden_rows("landing_zone_2d.txt")
    return np.array([[float(r[1]), float(r[2])] for r in rows], np.float32)


def _half_plane_landing(p, u, j):
    """p in L(u, j) by the geometry of Def. 6: the side of the perpendicular
    bisector of u-j that holds u, minus the closed ball around u of radius |u-j|."""
    mid = (u + j) / 2.0
    side = float(np.dot(p - mid, u - j)) > 0.0
    outside = float(np.linalg.norm(p - u)) > float(np.linalg.norm(j - u))
    return side and outside


def test_landing_zone_2d_hand_case(oracle_mod):
    O = oracle_mod
    X = _lz_points()
    A = np.zeros((len(X), 1), np.uint8)
    for cands, R, want in (([1, 2, 3, 4, 5, 6], 8, [1, 2, 3, 5]),
                           ([1, 2, 3, 4, 5, 6], 3, [1, 2, 3]),
                           ([1, 2, 3, 4, 5, 6, 7], 8, [1, 2, 3, 5])):
        cand = -np.ones((len(X), len(cands)), np.int64)
        cand[0] = cands
        nbr, deg = O.edge_select(X, A, cand, R, weights=(1.0, 0.0))
        got = [int(v) for v in nbr[0] if v >= 0]
        assert got == want
        assert deg[0] == len(want)


def test_landing_zone_matches_geometry_on_random_2d(oracle_mod):
    O = oracle_mod
    r = np.random.default_rng(4)
    for trial in range(30):
        X = r.standard_normal((40, 2)).astype(np.float32)
        A = np.zeros((40, 1), np.uint8)
        cand = -np.ones((40, 39), np.int64)
        cand[0] = np.arange(1, 40)
        nbr, _ = O.edge_select(X, A, cand, 10, weights=(1.0, 0.0))
        # rebuild N(0) with the half-plane geometry and the paper's steps
        Xd = X.astype(np.float64)
        order = sorted(range(1, 40), key=lambda i: (float(np.linalg.norm(Xd[i] - Xd[0])), i))
        sel = [order[0]]
        for p in order[1:]:
            if len(sel) == 10:
                break
            if all(_half_plane_landing(Xd[p], Xd[0], Xd[j]) for j in sel):
                sel.append(p)
        assert [int(v) for v in nbr[0] if v >= 0] == sel


def test_edge_select_invariants(oracle_mod):
    O = oracle_mod
    w = synth.int_valued(600, 1, 16, seed=12)
    cand, g = O.knn(w.X, w.A, 24, prec=O.F32)
    nbr, deg = O.edge_select(w.X, w.A, cand, 8, prec=O.F32)
    for u in range(0, 600, 7):
        row = [int(v) for v in nbr[u] if v >= 0]
        assert len(row) == deg[u] <= 8
        assert row[0] == cand[u, 0]  # step (2): the nearest candidate always joins
        assert len(set(row)) == len(row) and u not in row
        # every later neighbour p is closer to u than to any earlier neighbour j
        for a in range(len(row)):
            for b in range(a):
                p, j = row[a], row[b]
                gpu_ = O.gamma(O.delta(w.X[p], w.X[u], O.F32), O.chi(w.A[p], w.A[u]), w.m, prec=O.F32)
                gpj = O.gamma(O.delta(w.X[p], w.X[j], O.F32), O.chi(w.A[p], w.A[j]), w.m, prec=O.F32)
                assert gpu_ < gpj


def test_reverse_candidates_hand_case(oracle_mod):
    nbr = np.array([[1, 2, -1], [2, -1, -1], [0, 1, -1], [1, 0, 2]])
    out = oracle_mod.reverse_candidates(nbr, cap=2)
    assert out.tolist() == [[1, 2, 3, -1, -1], [2, 0, 3, -1, -1], [0, 1, 3, -1, -1],
                            [1, 0, 2, -1, -1]]


# ------------------------------------------------------------------ Alg. 2
def _complete_graph(n):
    return np.array([[j for j in range(n) if j != i] for i in range(n)], np.int64)


def test_search_complete_graph_is_exact(oracle_mod):
    O = oracle_mod
    w = synth.c1(N=30, nq=12, d=8, cards=(2, 3), seed=13)
    G = _complete_graph(30)
    ref, rg, _ = O.fused_topk(w.X, w.A, w.Qv, w.QA, 5, prec=O.F32)
    for h in (1, 2, 29):
        for ef in (5, 8, 30):
            r = O.search(w.X, w.A, G, w.Qv, w.QA, 5, ef, h=h, seed=3)
            assert (r["ids"] == ref).all(), (h, ef)
            assert np.array_equal(r["gamma"], rg)
            assert (r["status"] == 0).all()


def _reachable(nbr, seeds):
    seen, stack = set(seeds), list(seeds)
    while stack:
        u = stack.pop()
        for v in nbr[u]:
            if v >= 0 and v not in seen:
                seen.add(int(v))
                stack.append(int(v))
    return seen


def _seed_ids(O, seed, q, N, want=32):
    """Seed set B of the stated reading: first distinct ids of the splitmix64
    stream started at seed ^ mix64(q), reduced mod N, at most 64 draws."""
    seeds = []
    for x in O.splitmix64_stream(seed ^ O.mix64(q), 64):
        v = x % N
        if v not in seeds:
            seeds.append(v)
        if len(seeds) == want:
            break
    return seeds


def test_search_ef_ge_N_equals_brute_force_on_reachable_set(oracle_mod):
    O = oracle_mod
    w = synth.int_valued(250, 15, 16, seed=14)
    nbr, _, _ = O.build_graph(w.X, w.A, R=6, K=12)
    N, k = 250, 7
    r = O.search(w.X, w.A, nbr, w.Qv, w.QA, k, N, h=1, seed=99)
    for q in range(w.nq):
        reach = np.array(sorted(_reachable(nbr, _seed_ids(O, 99, q, N))))
        ids, _, _ = O.fused_topk(w.X[reach], w.A[reach], w.Qv[q:q + 1], w.QA[q:q + 1], k,
                                 prec=O.F32)
        assert list(r["ids"][q]) == list(reach[ids[0]])


def test_search_greedy_path_graph(oracle_mod):
    O = oracle_mod
    # 1-D chain 0-1-...-9 with x_i = i; ef = 1 greedy walk must end at the vertex
    # nearest the query, whatever the seed
    X = np.arange(10, dtype=np.float32)[:, None]
    A = np.zeros((10, 1), np.uint8)
    nbr = np.array([[i - 1 if i > 0 else -1, i + 1 if i < 9 else -1] for i in range(10)])
    for qx in (0.1, 3.4, 8.9):
        r = O.search(X, A, nbr, np.array([[qx]], np.float32), np.zeros((1, 1), np.uint8), 1, 1,
                     seed=7)
        assert r["ids"][0, 0] == int(round(qx))


def test_search_iteration_cap_reports_status(oracle_mod):
    O = oracle_mod
    w = synth.c1(N=200, nq=3, d=8, seed=15)
    nbr, _, _ = O.build_graph(w.X, w.A, R=8, K=16)
    r = O.search(w.X, w.A, nbr, w.Qv, w.QA, 4, 16, max_iters=0)
    assert (r["status"] == O.ITER_LIMIT).all() and (r["expansions"] == 0).all()
    assert (r["ndc"] == 16).all()  # only the seeds were evaluated
    r = O.search(w.X, w.A, nbr, w.Qv, w.QA, 4, 16, max_iters=1 << 20)
    assert (r["status"] == 0).all()


def test_search_recall_grows_with_ef(oracle_mod):
    O = oracle_mod
    w = synth.int_valued(2000, 60, 32, seed=16)
    nbr, _, _ = O.build_graph(w.X, w.A, R=16, K=32, weights=(1.0, 10000.0))
    ref, _, _ = O.fused_topk(w.X, w.A, w.Qv, w.QA, 10, weights=(1.0, 10000.0), prec=O.F32)
    rec = [O.recall(O.search(w.X, w.A, nbr, w.Qv, w.QA, 10, ef, weights=(1.0, 10000.0))["ids"],
                    ref) for ef in (10, 40, 160)]
    assert rec[0] <= rec[1] + 0.02 and rec[1] <= rec[2] + 0.02
    assert rec[2] > 0.9


# ------------------------------------------------------------------ Eq. 3
def test_recall_definitions(oracle_mod):
    O = oracle_mod
    assert O.recall([[1, 2, 3]], [[3, 2, 9]]) == pytest.approx(2 / 3)
    A = np.array([[0], [1], [0], [0]], np.uint8)
    QA = np.array([[0], [0]], np.uint8)
    found = np.array([[0, 1], [2, 3]])
    truth = np.array([[0, 2], [2, -1]])
    r, excl = O.hybrid_recall(found, A, QA, truth, np.array([3, 1]))
    # q0: matching returned {0}; hits {0} of min(2,3)=2 -> 0.5; q1: {2,3} & {2} -> 1/1
    assert r == pytest.approx(0.75) and excl == 0
    r, excl = O.hybrid_recall(found, A, QA, truth, np.array([0, 1]))
    assert excl == 1 and r == 1.0
    assert math.isfinite(r)


# ------------------------------------------------------------------ reduced-precision copies
def test_bf16_rounding_follows_the_format(oracle_mod):
    O = oracle_mod
    for x in (0.0, 1.0, -2.5, 255.0, 0.15625, 3.0e38):
        # values with at most 8 significant bits are representable and unchanged
        if x in (0.0, 1.0, -2.5, 255.0, 0.15625):
            assert O.round_bf16(x) == x
    assert O.round_bf16(1 + 2**-8) == 1.0                  # halfway: to even (1.0)
    assert O.round_bf16(1 + 3 * 2**-8) == 1 + 2**-6        # halfway: to even (1 + 2^-6)
    assert O.round_bf16(1 + 2**-8 + 2**-12) == 1 + 2**-7   # above halfway: up
    assert O.round_bf16(-(1 + 2**-8 + 2**-12)) == -(1 + 2**-7)


def test_row_rounding_matches_torch_bf16_and_e4m3(oracle_mod):
    # the array form used for candidate sets on rounded rows against an independent
    # library conversion (torch rounds f32 to bf16 and to e4m3 to nearest, ties to even)
    O = oracle_mod
    rng = np.random.default_rng(66)
    X = np.concatenate([rng.standard_normal(4000).astype(np.float32),
                        (rng.standard_normal(2000) * 100).astype(np.float32),
                        (rng.standard_normal(2000) * 1e-3).astype(np.float32)]).reshape(80, 100)
    b = O.round_rows(X, O.ROUND_BF16)
    assert np.array_equal(b, torch.from_numpy(X).to(torch.bfloat16).float().numpy())
    assert np.array_equal(b.ravel()[:50], np.array([O.round_bf16(x) for x in X.ravel()[:50]],
                                                   np.float32))
    inr = np.clip(X, -440, 440)  # torch's e4m3 conversion does not saturate; stay in range
    e = O.round_rows(inr, O.ROUND_E4M3)
    assert np.array_equal(e, torch.from_numpy(inr).to(torch.float8_e4m3fn).float().numpy())


def test_f16_rounding_matches_numpy_half(oracle_mod):
    # binary16 by its definition against numpy's conversion (round to nearest even),
    # across normals, subnormals, halfway cases and overflow
    O = oracle_mod
    rng = np.random.default_rng(73)
    X = np.concatenate([rng.standard_normal(3000) * s for s in (1.0, 1e3, 3e4, 1e-5, 1e-7)]
                       + [np.array([65504.0, 65519.0, 65520.0, 70000.0, -65520.0, 2.0 ** -24,
                                    2.0 ** -25, 3 * 2.0 ** -26, 1 + 2.0 ** -11,
                                    1 + 3 * 2.0 ** -11, 0.0, -0.0])]).astype(np.float32)
    got = O.round_rows(X, O.ROUND_F16)
    with np.errstate(over="ignore"):  # the values beyond 65504 round to infinity
        want = X.astype(np.float16).astype(np.float32)
    assert np.array_equal(got, want)
    assert np.array_equal(np.signbit(got), np.signbit(want))


def test_knn_on_rounded_rows_is_knn_of_the_rounded_copy(oracle_mod):
    O = oracle_mod
    w = synth.c1(N=300, nq=1, d=24, seed=67)
    a, ga = O.knn(w.X, w.A, 8, vec_round=O.ROUND_BF16)
    b, gb = O.knn(O.round_rows(w.X, O.ROUND_BF16), w.A, 8)
    assert (a == b).all() and np.array_equal(ga, gb)
    c, _ = O.knn(w.X, w.A, 8)
    assert not np.array_equal(ga, O.knn(w.X, w.A, 8)[1])  # the rounding is not a no-op
    assert (a[:, 0] != np.arange(300)).all() and c.shape == a.shape


def test_e4m3_rounding_follows_the_format(oracle_mod):
    O = oracle_mod
    for x in (0.0, 1.0, 1.125, 16.0, 18.0, 448.0, -240.0, 2**-6, 2**-9, 3 * 2**-9):
        assert O.round_e4m3(x) == x                        # representable values
    assert O.round_e4m3(17.0) == 16.0                      # halfway 16|18: to even
    assert O.round_e4m3(19.0) == 20.0                      # halfway 18|20: to even
    assert O.round_e4m3(1.0625) == 1.0                     # halfway 1|1.125: to even
    assert O.round_e4m3(470.0) == 448.0 and O.round_e4m3(-1e6) == -448.0   # saturation
    assert O.round_e4m3(2**-10) == 0.0                     # half the smallest subnormal: even
    assert O.round_e4m3(3 * 2**-10) == 2**-8               # halfway 2^-9|2^-8: to even
    assert O.round_e4m3(2**-10 + 2**-14) == 2**-9          # above halfway: up


def test_reduced_precision_search_equals_plain_on_exact_data(oracle_mod):
    O = oracle_mod
    # integer components 0..255 are exact in bf16: scoring with the copy changes nothing
    w = synth.int_valued(600, 20, 16, seed=17)
    nbr, _, _ = O.build_graph(w.X, w.A, R=8, K=16)
    a = O.search(w.X, w.A, nbr, w.Qv, w.QA, 5, 20, seed=3)
    b = O.search(w.X, w.A, nbr, w.Qv, w.QA, 5, 20, seed=3, vec_round=O.ROUND_BF16)
    c = O.search(w.X, w.A, nbr, w.Qv, w.QA, 5, 20, seed=3, vec_round=O.ROUND_BF16, rerank=True)
    assert (a["ids"] == b["ids"]).all() and (a["ids"] == c["ids"]).all()
    # fp8 scoring differs, and the re-rank returns exact Gamma values for its ids
    d = O.search(w.X, w.A, nbr, w.Qv, w.QA, 5, 20, seed=3, vec_round=O.ROUND_E4M3, rerank=True)
    for q in range(w.nq):
        for j, i in enumerate(d["ids"][q]):
            g = O.gamma(O.delta(w.Qv[q], w.X[i], O.F32), O.chi(w.QA[q], w.A[i]), w.m, prec=O.F32)
            assert d["gamma"][q, j] == g
        assert all(np.diff(d["gamma"][q]) >= 0)


# ------------------------------------------------------------------ learned stop model (oracle)
def test_mlp_zero_weights_closed_form():
    from oracle import mlp

    p = np.zeros(mlp.N_PARAMS)
    X = np.random.default_rng(0).standard_normal((50, 8))
    y = (np.arange(50) % 3 == 0).astype(float)
    loss, g = mlp.loss_and_grad(p, X, y)
    assert loss == pytest.approx(np.log(2.0), rel=1e-15)   # sigmoid(0) = 1/2
    W1, b1, W2, b2 = mlp.unpack(g)
    assert b2 == pytest.approx(np.mean(0.5 - y), rel=1e-14)
    assert not W1.any() and not b1.any() and not W2.any()   # h = 0 and W2 = 0


def test_mlp_gradient_matches_finite_differences():
    from oracle import mlp

    r = np.random.default_rng(1)
    p = r.standard_normal(mlp.N_PARAMS) * 0.3
    X = r.standard_normal((40, 8))
    y = (r.random(40) < 0.4).astype(float)
    _, g = mlp.loss_and_grad(p, X, y)
    eps = 1e-6
    for i in r.choice(mlp.N_PARAMS, 60, replace=False):
        e = np.zeros_like(p)
        e[i] = eps
        lp, _ = mlp.loss_and_grad(p + e, X, y)
        lm, _ = mlp.loss_and_grad(p - e, X, y)
        assert g[i] == pytest.approx((lp - lm) / (2 * eps), rel=1e-5, abs=1e-9)


def test_mlp_forward_hand_case():
    from oracle import mlp

    W1 = np.zeros((8, 64))
    W1[0, 0], W1[1, 0], W1[2, 1] = 2.0, -1.0, 1.0
    b1 = np.zeros(64)
    b1[1] = -0.5
    W2 = np.zeros(64)
    W2[0], W2[1] = 1.5, -2.0
    p = mlp.pack(W1, b1, W2, 0.25)
    x = np.array([[1.0, 0.5, 2.0, 0, 0, 0, 0, 0], [-1.0, 0.0, 0.2, 0, 0, 0, 0, 0]])
    # row 0: h0 = relu(2 - .5) = 1.5, h1 = relu(2 - .5) = 1.5 -> 1.5*1.5 - 2*1.5 + .25 = -0.5
    # row 1: h0 = relu(-2) = 0, h1 = relu(.2 - .5) = 0 -> 0.25
    assert np.allclose(mlp.forward(p, x), [-0.5, 0.25], rtol=0, atol=1e-15)


# ------------------------------------------------------------------ curves i and ii (Sec. 6.5)
def test_harmonic_curve_i_is_the_harmonic_mean_and_vanishes_at_chi_zero(oracle_mod):
    O = oracle_mod
    # Gamma = 2 delta chi / (delta + chi); the paper's stated defect: chi = 0 gives 0
    assert O.gamma(3.0, 1, 3, "harmonic") == pytest.approx(1.5, rel=0, abs=1e-15)
    assert O.gamma(1.0, 3, 3, "harmonic") == pytest.approx(1.5, rel=0, abs=1e-15)  # symmetric
    for d in (0.0, 0.5, 7.0, 1e6):
        assert O.gamma(d, 0, 3, "harmonic") == 0.0
        assert O.gamma(d, 0, 3, "harmonic", O.F32) == 0.0


def test_harmonic_curve_ii_adjusts_chi(oracle_mod):
    O = oracle_mod
    # chi -> 1 for chi = 0 and c * chi otherwise (c = 100)
    for d in (0.25, 3.0, 40.0):
        assert O.gamma(d, 0, 3, ("harmonic", 100.0)) == pytest.approx(2 * d / (d + 1), rel=1e-15)
        assert O.gamma(d, 2, 3, ("harmonic", 100.0)) == pytest.approx(400 * d / (d + 200),
                                                                        rel=1e-15)


@pytest.mark.parametrize("c", [0.0, 100.0])
def test_harmonic_bounds_monotonicity_and_f32(oracle_mod, c):
    O = oracle_mod
    w = ("harmonic", c) if c else "harmonic"
    rng = np.random.default_rng(5)
    for d in rng.random(200) * 50:
        prev = -1.0
        for chi in range(4):
            h = chi if c == 0 else (1.0 if chi == 0 else c * chi)
            g = O.gamma(d, chi, 3, w)
            # a harmonic mean lies between the smaller value and twice it
            assert min(d, h) - 1e-12 <= g <= 2 * min(d, h) + 1e-12
            assert g >= prev  # non-decreasing in chi
            prev = g
            g32 = O.gamma(float(np.float32(d)), chi, 3, w, O.F32)
            assert g32 == pytest.approx(O.gamma(float(np.float32(d)), chi, 3, w), rel=1e-6,
                                        abs=1e-30)
        assert O.gamma(d, 1, 3, w) <= O.gamma(d + 1.0, 1, 3, w)  # non-decreasing in delta


def test_curve_i_brute_force_returns_the_smallest_matching_ids(oracle_mod):
    O = oracle_mod
    # every exact attribute match has Gamma 0, so the top-k are the k smallest matching
    # ids (ties by id) whenever there are at least k matches
    w = synth.int_valued(600, 8, 8, cards=(2, 3), seed=12)
    ids, g, chi = O.fused_topk(w.X, w.A, w.Qv, w.QA, 5, weights="harmonic", prec=O.F32)
    for q in range(w.nq):
        match = np.nonzero((w.A == w.QA[q]).all(axis=1))[0]
        assert len(match) >= 5
        assert (ids[q] == match[:5]).all() and (g[q] == 0).all() and (chi[q] == 0).all()


# ------------------------------------------------------------------ incremental build (NPG_nsw)
def test_nsw_waves_cover_every_vertex_once(oracle_mod):
    O = oracle_mod
    for N, cap in ((1, 8), (2, 8), (100, 8), (1000, 64)):
        waves = O.nsw_waves(N, cap)
        covered = [v for s, e in waves for v in range(s, e)]
        assert covered == list(range(1, N))
        assert all(e - s <= min(s, cap) for s, e in waves)


def test_nsw_insertion_search_is_exhaustive_on_a_small_prefix(oracle_mod):
    # with waves of one vertex and every earlier vertex a seed (s <= 32), each insertion
    # evaluates all of [0, v): its candidates are the exact fused top-L of the prefix
    O = oracle_mod
    w = synth.int_valued(33, 1, 8, cards=(2, 3), seed=21)
    for weights in (None, (1.0, 10000.0)):
        _, steps = O.build_nsw(w.X, w.A, R=4, L=40, weights=weights, wave_max=1, trace=True)
        assert len(steps) == 32
        for W, cand in steps:
            v = int(W[0])
            ref, _, _ = O.fused_topk(w.X[:v], w.A[:v], w.X[v:v + 1], w.A[v:v + 1], min(40, v),
                                     weights=weights, prec=O.F32)
            assert (cand[0, :v] == ref[0]).all() and (cand[0, v:] == -1).all()


def test_nsw_graph_is_well_formed(oracle_mod):
    O = oracle_mod
    w = synth.int_valued(400, 1, 8, cards=(2, 3), seed=22)
    nbr = O.build_nsw(w.X, w.A, R=8, L=24, wave_max=16)
    assert nbr.shape == (400, 8)
    for u in range(400):
        row = nbr[u][nbr[u] >= 0]
        # vertex 0 gains its edges from later insertions; every other vertex keeps at least
        # the nearest vertex its search found
        assert len(row) >= 1
        assert u not in row and len(set(row.tolist())) == len(row) and (row < 400).all()


def test_nsw_attribute_entry_picks_earlier_matches(oracle_mod):
    O = oracle_mod
    A = np.array([[0, 1], [1, 1], [0, 1], [0, 0], [0, 1], [1, 1]], np.uint8)
    # vertex 4 (0, 1) among [0, 4): matches 0 and 2
    assert O.nsw_attribute_seeds(4, 4, A, 0)[:3] == [0, 2, -1]
    # vertex 3 (0, 0) has no earlier match: the id rule
    assert O.nsw_attribute_seeds(3, 3, A, 9) == O.nsw_seeds(3, 3, 9)
    # evenly spaced when there are more matches than seeds
    big = np.zeros((100, 1), np.uint8)
    assert O.nsw_attribute_seeds(99, 96, big, 0, n=4) == [0, 24, 48, 72]


def test_nearest_attribute_entry_seeds_are_the_nearest_matches(oracle_mod):
    # with |P| <= 256 every match is sampled, so the seed pool holds the min(ef, 32)
    # nearest matches; with no expansion the top-k is the exact filtered top-k
    O = oracle_mod
    w = synth.int_valued(3000, 40, 16, cards=(3, 5, 4), seed=23)
    CONST = (1.0, 10000.0)
    nbr = np.full((w.N, 4), -1, np.int64)
    r = O.search(w.X, w.A, nbr, w.Qv, w.QA, 10, 32, weights=CONST, max_iters=0,
                 seed_mode=O.SEED_ATTRIBUTE_NEAR)
    ref, _, P = O.filtered_topk(w.X, w.A, w.Qv, w.QA, 10, prec=O.F32)
    checked = 0
    for q in range(w.nq):
        if 10 <= P[q] <= 256:
            assert (r["ids"][q] == ref[q]).all(), q
            checked += 1
    assert checked >= 20


# ------------------------------------------------------------------ partial constraints
def test_chi_query_wildcard_hand_cases(oracle_mod):
    O = oracle_mod
    q = np.array([1, 255, 3, 255], np.uint8)
    assert O.chi_query(q, np.array([1, 7, 3, 0], np.uint8), 255) == 0   # open positions
    assert O.chi_query(q, np.array([2, 255, 4, 255], np.uint8), 255) == 2
    assert O.chi_query(q, np.array([1, 7, 4, 0], np.uint8), 255) == 1
    # without a wildcard 255 is an ordinary code
    assert O.chi_query(q, np.array([1, 7, 3, 0], np.uint8)) == 2
    assert O.chi_query(q, np.array([1, 255, 3, 255], np.uint8)) == 0
    # a different wildcard code
    assert O.chi_query(np.array([9, 4], np.uint8), np.array([5, 4], np.uint8), 9) == 0


def test_fully_open_query_is_plain_l2(oracle_mod):
    # every position open: chi = 0 for every object, so Gamma = w_v * delta and the
    # exact fused top-k is the L2 top-k by (delta, id), computed here with numpy
    O = oracle_mod
    w = synth.int_valued(500, 20, 12, cards=(3, 4, 5), seed=57)
    QA = np.full_like(w.QA, 255)
    d2 = ((w.Qv[:, None, :].astype(np.int64) - w.X[None, :, :].astype(np.int64)) ** 2).sum(-1)
    want = np.array([np.lexsort((np.arange(w.N), d2[q]))[:10] for q in range(w.nq)])
    for wts in (None, (1.0, 10000.0)):
        ids, g, ch = O.fused_topk(w.X, w.A, w.Qv, QA, 10, weights=wts, prec=O.F32,
                                  wildcard=255)
        assert (ids == want).all()
        assert (ch == 0).all()
        assert np.array_equal(g, np.sqrt(np.take_along_axis(d2, want, 1).astype(np.float32)))


def test_partially_open_filter_matches_constrained_columns(oracle_mod):
    # the hybrid ground truth under a partial constraint: the objects equal on the
    # constrained columns only, by (delta, id), computed here with numpy
    O = oracle_mod
    w = synth.int_valued(800, 30, 8, cards=(3, 4, 5), seed=58)
    QA = w.QA.copy()
    QA[::2, 1] = 255
    QA[::3, 0] = 255
    ids, dl, P = O.filtered_topk(w.X, w.A, w.Qv, QA, 10, prec=O.F32, wildcard=255)
    d2 = ((w.Qv[:, None, :].astype(np.int64) - w.X[None, :, :].astype(np.int64)) ** 2).sum(-1)
    for q in range(w.nq):
        cols = QA[q] != 255
        ok = np.flatnonzero((w.A[:, cols] == QA[q, cols]).all(axis=1))
        assert P[q] == ok.size
        order = ok[np.lexsort((ok, d2[q, ok]))][:10]
        assert (ids[q, :order.size] == order).all() and (ids[q, order.size:] == -1).all()


def test_search_with_open_positions(oracle_mod):
    O = oracle_mod
    w = synth.c1(N=30, nq=12, d=8, cards=(2, 3), seed=13)
    QA = w.QA.copy()
    QA[::2, 0] = 255
    G = _complete_graph(30)
    ref, rg, _ = O.fused_topk(w.X, w.A, w.Qv, QA, 5, prec=O.F32, wildcard=255)
    for ef in (5, 30):
        r = O.search(w.X, w.A, G, w.Qv, QA, 5, ef, seed=3, wildcard=255)
        assert (r["ids"] == ref).all() and np.array_equal(r["gamma"], rg)


def test_open_query_seeds_come_from_the_completion_runs(oracle_mod):
    # with no expansion the result is the k best seeds; the seeds of an open query are
    # mode 1's evenly spaced picks over the runs of its completions, listed here with
    # itertools in completion order (lowest open position fastest)
    import itertools

    O = oracle_mod
    w = synth.int_valued(400, 24, 6, cards=(3, 4, 2), seed=59, zipf=False)
    QA = w.QA.copy()
    QA[:, 0] = 255
    QA[1::2, 2] = 255
    CONST = (1.0, 10000.0)
    nbr = np.full((w.N, 2), -1, np.int64)
    for ef in (8, 32):
        r = O.search(w.X, w.A, nbr, w.Qv, QA, 5, ef, seed=3, wildcard=255, max_iters=0,
                     weights=CONST, seed_mode=O.SEED_ATTRIBUTE, prec=O.F32)
        amax = w.A.max(axis=0)
        for q in range(w.nq):
            opn = [j for j in range(w.m) if QA[q, j] == 255]
            members = []
            for digits in itertools.product(*[range(amax[j] + 1) for j in reversed(opn)]):
                tup = QA[q].astype(int).copy()
                for j, dgt in zip(reversed(opn), digits):
                    tup[j] = dgt
                members += np.flatnonzero((w.A == tup).all(axis=1)).tolist()
            c = len(members)
            S = min(ef, 32, c)
            seeds = [members[(j * c) // S] for j in range(S)]
            g = [O.gamma(O.delta(w.Qv[q], w.X[v], O.F32), O.chi_query(QA[q], w.A[v], 255), w.m,
                         CONST, O.F32) for v in seeds]
            want = [v for _, v in sorted(zip(g, seeds))][:5]
            assert list(r["ids"][q][: len(want)]) == want, (ef, q)


def test_open_query_nearest_seeds_are_the_nearest_matches(oracle_mod):
    # mode 3 on an open query: with |P| <= 256 every member of the completion runs is
    # ranked, so with no expansion the top-k is the exact filtered top-k of the partial
    # constraint (itself pinned against numpy above)
    O = oracle_mod
    w = synth.int_valued(3000, 40, 16, cards=(3, 5, 4), seed=61)
    QA = w.QA.copy()
    QA[:, 0] = 255
    CONST = (1.0, 10000.0)
    nbr = np.full((w.N, 4), -1, np.int64)
    r = O.search(w.X, w.A, nbr, w.Qv, QA, 10, 32, weights=CONST, max_iters=0, wildcard=255,
                 seed_mode=O.SEED_ATTRIBUTE_NEAR)
    ref, _, P = O.filtered_topk(w.X, w.A, w.Qv, QA, 10, prec=O.F32, wildcard=255)
    checked = 0
    for q in range(w.nq):
        if 10 <= P[q] <= 256:
            assert (r["ids"][q] == ref[q]).all(), q
            checked += 1
    assert checked >= 20


# ------------------------------------------------------------------ seed set B (closed queries)
_M64 = (1 << 64) - 1


def _splitmix64_py(state, n):
    """First n outputs of Vigna's splitmix64 from ``state``, written out in Python
    (add the golden gamma, then the two xor-shift-multiply rounds and a final xor-shift)."""
    out = []
    for _ in range(n):
        state = (state + 0x9E3779B97F4A7C15) & _M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        out.append(z ^ (z >> 31))
    return out


def _mix64_py(z):
    """The finaliser of splitmix64 applied to z (one output from state z - gamma)."""
    return _splitmix64_py((z - 0x9E3779B97F4A7C15) & _M64, 1)[0]


def _seed_pool_f32(Qv, QA, X, A, q, seeds, wl):
    """(Gamma, id) of the seeds in f32 from integer arithmetic: delta^2 is an exact integer
    below 2^24, delta = its correctly rounded square root, Gamma = 1 * delta + w_l * chi with
    one f32 rounding (constant weights); with w_l = None the proportional form, which for
    chi = 0 is delta itself."""
    recs = []
    for v in seeds:
        d2 = int(((Qv[q].astype(np.int64) - X[v].astype(np.int64)) ** 2).sum())
        dl = np.sqrt(np.float32(d2))
        ch = int((A[v] != QA[q]).sum())
        if wl is None:
            assert ch == 0
            g = dl
        else:
            g = np.float32(dl + np.float32(np.float32(wl) * np.float32(ch)))
        recs.append((float(g), int(v)))
    return sorted(recs)


@pytest.mark.parametrize("weights", [None, (1.0, 10000.0)])
def test_closed_query_attribute_entry_seeds_are_evenly_spaced_matches(oracle_mod, weights):
    # Alg. 2's seed set B under the attribute-entry reading, for queries that constrain
    # every attribute: P = the objects equal to the query on all attributes, ascending
    # ids; S = min(ef, 32, |P|) seeds P[floor(j |P| / S)]; |P| = 0 falls back to the first
    # min(ef, 32) distinct ids of splitmix64(seed ^ mix64(q)) mod N (at most 64 draws).
    # With an empty graph and no expansion the pool is exactly B, returned by (Gamma, id).
    O = oracle_mod
    w = synth.int_valued(600, 40, 6, cards=(3, 4, 2), seed=63, zipf=False)
    QA = w.QA.copy()
    QA[::5, 1] = 7  # no object has code 7: |P| = 0 for every fifth query
    wl = None if weights is None else weights[1]
    nbr = np.full((w.N, 3), -1, np.int64)
    seed = 0x5EED
    for ef in (8, 32, 48):
        r = O.search(w.X, w.A, nbr, w.Qv, QA, ef, ef, seed=seed, max_iters=0, weights=weights,
                     seed_mode=O.SEED_ATTRIBUTE, prec=O.F32)
        for q in range(w.nq):
            P = np.flatnonzero((w.A == QA[q]).all(axis=1))
            c = P.size
            if c > 0:
                S = min(ef, 32, c)
                B = [int(P[(j * c) // S]) for j in range(S)]
            else:
                want, B = min(ef, 32), []
                for x in _splitmix64_py((seed ^ _mix64_py(q)) & _M64, 64):
                    v = x % w.N
                    if v not in B:
                        B.append(v)
                    if len(B) == want:
                        break
            if c == 0 and wl is None:  # proportional weights, chi > 0: the set of ids
                assert sorted(v for v in r["ids"][q] if v >= 0) == sorted(B), (ef, q)
                continue
            expect = _seed_pool_f32(w.Qv, QA, w.X, w.A, q, B, wl)
            assert [v for _, v in expect] == list(r["ids"][q][:len(B)]), (ef, q)
            assert (r["ids"][q][len(B):] == -1).all(), (ef, q)
            assert np.array_equal(np.array([g for g, _ in expect]),
                                  r["gamma"][q][:len(B)].astype(np.float32).astype(np.float64))
            assert r["ndc"][q] == len(B)


def test_nearest_attribute_entry_seeds_sample_large_match_sets(oracle_mod):
    # the nearest-entry rule with |P| > 256: the M = 256 members P[floor(j |P| / M)] are
    # ranked by (delta^2, id) and the min(ef, 32) first are the seeds
    O = oracle_mod
    w = synth.int_valued(4000, 30, 8, cards=(2, 2, 2), seed=64, zipf=False)
    CONST = (1.0, 10000.0)
    nbr = np.full((w.N, 3), -1, np.int64)
    for ef in (10, 32):
        r = O.search(w.X, w.A, nbr, w.Qv, w.QA, ef, ef, weights=CONST, max_iters=0,
                     seed_mode=O.SEED_ATTRIBUTE_NEAR, prec=O.F32)
        for q in range(w.nq):
            P = np.flatnonzero((w.A == w.QA[q]).all(axis=1))
            c = P.size
            assert c > 256
            sample = P[[(j * c) // 256 for j in range(256)]]
            d2 = ((w.Qv[q].astype(np.int64) - w.X[sample].astype(np.int64)) ** 2).sum(-1)
            B = sample[np.lexsort((sample, d2))][:min(ef, 32)]
            expect = _seed_pool_f32(w.Qv, w.QA, w.X, w.A, q, B, 10000.0)
            assert [v for _, v in expect] == list(r["ids"][q]), (ef, q)


# ------------------------------------------------------------------ NPG_nsw: serial limit
def _serial_nsw(O, X, A, R, L, weights, seed, entry):
    """NPG_nsw as Sec. 4.3 states it, one object at a time: object v searches the graph
    of the objects inserted before it for its L nearest (Alg. 2, k = ef = L), keeps a
    landing-zone selection of them as N(v) (Def. 6), and every u in N(v) re-selects from
    N(u) plus v."""
    N = X.shape[0]
    nbr = np.full((N, R), -1, np.int64)
    for v in range(1, N):
        B = O.nsw_attribute_seeds(v, v, A, seed) if entry else O.nsw_seeds(v, v, seed)
        r = O.search(X, A, nbr, X[v:v + 1], A[v:v + 1], L, L, seeds=np.array([B]),
                     weights=weights, prec=O.F32)
        row, _ = O.edge_select(X, A, r["ids"], R, weights=weights, prec=O.F32, rows=[v])
        nbr[v] = row[0]
        for u in row[0]:
            if u < 0:
                continue
            cu = np.full((1, R + 1), -1, np.int64)
            old = [x for x in nbr[u] if x >= 0]
            cu[0, :len(old) + 1] = old + [v]
            nbr[u] = O.edge_select(X, A, cu, R, weights=weights, prec=O.F32, rows=[u])[0][0]
    return nbr


@pytest.mark.parametrize("weights,entry", [(None, 0), ((1.0, 10000.0), 1)])
def test_nsw_single_vertex_waves_are_serial_insertion(oracle_mod, weights, entry):
    O = oracle_mod
    w = synth.int_valued(160, 1, 8, cards=(2, 3), seed=65)
    got = O.build_nsw(w.X, w.A, R=6, L=12, weights=weights, seed=11, wave_max=1, entry=entry)
    ref = _serial_nsw(O, w.X, w.A, 6, 12, weights, 11, entry)
    assert np.array_equal(got, ref)


# ------------------------------------------------------------------ entry cells, entry model
def test_cells_are_the_nearest_centroids_by_integer_delta(oracle_mod):
    O = oracle_mod
    w = synth.int_valued(900, 40, 12, seed=71)
    E = 37
    cid = O.cell_centroids(w.N, E)
    assert list(cid[:3]) == [0, 24, 48] and len(set(cid.tolist())) == E
    d2 = ((w.X[:, None, :].astype(np.int64) - w.X[None, cid, :].astype(np.int64)) ** 2).sum(-1)
    want = np.array([np.lexsort((np.arange(E), r))[0] for r in d2])
    assert (O.cells(w.X, E) == want).all()
    assert (O.cells(w.X, E)[cid] == np.arange(E)).all() or len(set(map(tuple, w.X[cid]))) < E
    q2 = ((w.Qv[:, None, :].astype(np.int64) - w.X[None, cid, :].astype(np.int64)) ** 2).sum(-1)
    near = O.nearest_cells(w.X, E, w.Qv, 4)
    for q in range(w.nq):
        assert list(near[q]) == list(np.lexsort((np.arange(E), q2[q]))[:4])


def test_cell_seeds_hand_case(oracle_mod):
    O = oracle_mod
    A = np.array([[0], [1], [0], [0], [1], [0], [0], [0]], np.uint8)
    cell_of = np.array([2, 0, 1, 2, 1, 1, 0, 2])
    QA = np.array([[0], [0], [1], [0]], np.uint8)
    chosen = np.array([[1, 2], [0, 1], [2, 0], [3, 0]])
    B = O.cell_seeds(A, QA, cell_of, chosen, ef=32)
    # q0: P = 0 2 3 5 6 7; cell 1 -> 2 5, cell 2 -> 0 3 7; S = 6 -> all five, then P[0]
    assert list(B[0][:6]) == [2, 5, 0, 3, 7, 0] and (B[0][6:] == -1).all()
    # q1: cell 0 -> 6, cell 1 -> 2 5; S = 6 -> then 3 evenly spaced of P: P[0], P[2], P[4]
    assert list(B[1][:6]) == [6, 2, 5, 0, 3, 6]
    # q2: P = 1 4; cell 2 none, cell 0 -> 1; S = 2 -> then P[0]
    assert list(B[2][:2]) == [1, 1] and (B[2][2:] == -1).all()
    # a small ef limits S; cells with no member of P give nothing
    B = O.cell_seeds(A, QA, cell_of, chosen, ef=3)
    assert list(B[3][:3]) == [6, 0, 5] and (B[3][3:] == -1).all()  # P[0], P[3]
    # no match: the random stream
    B = O.cell_seeds(A, np.array([[5]], np.uint8), cell_of, np.array([[0, 1]]), ef=4, seed=9)
    ref = []
    for x in _splitmix64_py((9 ^ _mix64_py(0)) & _M64, 64):
        if x % 8 not in ref:
            ref.append(x % 8)
        if len(ref) == 4:
            break
    assert list(B[0][:4]) == ref


def test_entry_model_zero_weights_and_gradient(oracle_mod):
    from oracle import mlp

    d, E = 6, 9
    p = np.zeros(mlp.entry_size(d, E))
    p[0] = 0.5
    rng = np.random.default_rng(72)
    Q, y = rng.standard_normal((13, d)), rng.integers(0, E, 13)
    loss, g = mlp.entry_loss_and_grad(p, Q, y, d, E)
    assert abs(loss - math.log(E)) < 1e-12  # uniform softmax
    # with zero weights only b2 has a gradient: mean(1/E - onehot)
    _, _, _, _, gb2 = mlp.entry_unpack(g, d, E)
    want = np.full(E, 1.0 / E) - np.bincount(y, minlength=E) / 13
    assert np.allclose(gb2, want)
    p = rng.standard_normal(p.size) * 0.3
    p[0] = 0.7
    loss, g = mlp.entry_loss_and_grad(p, Q, y, d, E)
    num = np.zeros_like(p)
    for i in range(1, p.size):
        e = np.zeros_like(p)
        e[i] = 1e-6
        num[i] = (mlp.entry_loss_and_grad(p + e, Q, y, d, E)[0] -
                  mlp.entry_loss_and_grad(p - e, Q, y, d, E)[0]) / 2e-6
    assert np.abs(num - g).max() < 1e-7 and g[0] == 0.0
    # forward: softmax of the logits reproduces the loss
    t = mlp.entry_forward(p, Q, d, E)
    lse = np.log(np.exp(t).sum(1))
    assert abs(np.mean(lse - t[np.arange(13), y]) - loss) < 1e-12
