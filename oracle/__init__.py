"""Plain CPU oracle of the NHQ hybrid-query path (arXiv 2203.13601).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.  It
shares no code with the CUDA library.  The arithmetic lives in ``nhq_oracle.c``
(plain serial C, see its header for the paper passage behind each function);
this module only compiles it with gcc and marshals numpy arrays.

Every function here follows a definition of the paper:

* ``delta`` / ``chi`` / ``gamma``  Eq. 1, Eq. 4-5, Eq. 6 (weights of Sec. 3.2)
* ``fused_topk``                   exact top-k by (Gamma, id) (Def. 2 with Gamma)
* ``filtered_topk``                hybrid ground truth of Sec. 6.1
* ``knn``                          candidate sets C(u) of Sec. 4.1 (exact K nearest)
* ``edge_select``                  landing-zone edge selection (Sec. 4.1, Def. 6)
* ``search``                       Alg. 2 joint pruning + two-stage routing (Sec. 4.2, 5.2)
* ``graph_quality``                Eq. 7
* ``recall`` / ``hybrid_recall``   Eq. 3 and its hybrid form (Sec. 6.1)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nhq_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

W_PROPORTIONAL = 0  # w_v = 1, w_l = delta / m  (Sec. 3.2, curve iv)
W_CONSTANT = 1      # w_v, w_l given             (Eq. 6, curve v)
W_HARMONIC = 3      # 2 delta h / (delta + h), h = chi (curve i) or 1 / c chi (curve ii)
F64 = 0
F32 = 1
ITER_LIMIT = 4

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            i64, i32, f64, u64 = C.c_int64, C.c_int, C.c_double, C.c_uint64
            lib.or_mix64.restype = u64
            lib.or_mix64.argtypes = [u64]
            lib.or_splitmix64_at.restype = u64
            lib.or_splitmix64_at.argtypes = [u64, u64]
            lib.or_delta64.restype = f64
            lib.or_delta64.argtypes = [P, P, i32]
            lib.or_delta32.restype = C.c_float
            lib.or_delta32.argtypes = [P, P, i32]
            lib.or_chi.restype = i32
            lib.or_chi.argtypes = [P, P, i32]
            lib.or_chi_query.restype = i32
            lib.or_chi_query.argtypes = [P, P, i32, i32]
            lib.or_gamma64.restype = f64
            lib.or_gamma64.argtypes = [f64, i32, i32, i32, f64, f64]
            lib.or_gamma32.restype = C.c_float
            lib.or_gamma32.argtypes = [C.c_float, i32, i32, i32, C.c_float, C.c_float]
            lib.or_fused_topk.restype = None
            lib.or_fused_topk.argtypes = [P, P, i64, i32, i32, P, P, i64, i32, i32, f64, f64, i32,
                                          P, P, P, i32]
            lib.or_filtered_topk.restype = None
            lib.or_filtered_topk.argtypes = [P, P, i64, i32, i32, P, P, i64, i32, i32, P, P, P,
                                             i32]
            lib.or_knn.restype = None
            lib.or_knn.argtypes = [P, P, i64, i32, i32, i32, i32, f64, f64, i32, P, i64, P, P]
            lib.or_edge_select.restype = None
            lib.or_edge_select.argtypes = [P, P, i64, i32, i32, P, i32, i32, i32, f64, f64, i32,
                                           P, i64, P, P]
            lib.or_reverse_candidates.restype = None
            lib.or_reverse_candidates.argtypes = [P, i64, i32, i32, P, i64, P]
            lib.or_graph_quality.restype = f64
            lib.or_graph_quality.argtypes = [P, i64, i32, P, i32]
            lib.or_search.restype = None
            lib.or_search.argtypes = [P, P, i64, i32, i32, P, i32, P, P, i64, i32, i32, i32, u64,
                                      i64, i32, f64, f64, i32, i32, P, i32, i32, i32, P, P, P, P,
                                      P, P, i32]
            lib.or_round_bf16.restype = C.c_float
            lib.or_round_bf16.argtypes = [C.c_float]
            lib.or_round_e4m3.restype = C.c_float
            lib.or_round_e4m3.argtypes = [C.c_float]
            lib.or_round_rows.restype = None
            lib.or_round_rows.argtypes = [P, i64, i32]
            _lib = lib
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _mode(weights):
    """weights: None / "proportional" -> Sec. 3.2 recommended form; (w_v, w_l) -> constant;
    "harmonic" -> curve i of Sec. 6.5; ("harmonic", c) -> curve ii with constant c."""
    if weights is None or weights == "proportional":
        return W_PROPORTIONAL, 1.0, 0.0
    if weights == "harmonic":
        return W_HARMONIC, 1.0, 0.0
    if weights[0] == "harmonic":
        return W_HARMONIC, 1.0, float(weights[1])
    wv, wl = weights
    return W_CONSTANT, float(wv), float(wl)


# ---------------------------------------------------------------- scalars
def mix64(z: int) -> int:
    return int(_L().or_mix64(C.c_uint64(z & (2**64 - 1))))


def splitmix64_stream(state: int, n: int) -> list:
    """First n outputs of splitmix64 started from ``state``."""
    return [int(_L().or_splitmix64_at(C.c_uint64(state & (2**64 - 1)), j)) for j in range(n)]


def delta(x, y, prec=F64) -> float:
    x, y = _f32(x), _f32(y)
    f = _L().or_delta32 if prec == F32 else _L().or_delta64
    return float(f(_p(x), _p(y), x.shape[0]))


def chi(a, b) -> int:
    a, b = _u8(a), _u8(b)
    return int(_L().or_chi(_p(a), _p(b), a.shape[0]))


def chi_query(qa, a, wildcard=None) -> int:
    """chi of a query against an object; with ``wildcard`` (a code 0..255), query
    positions holding that code are unconstrained and never count."""
    qa, a = _u8(qa), _u8(a)
    return int(_L().or_chi_query(_p(qa), _p(a), qa.shape[0], _wild(wildcard)))


def _wild(wildcard):
    return -1 if wildcard is None else int(wildcard)


def gamma(delta_value, chi_value, m, weights=None, prec=F64) -> float:
    mode, wv, wl = _mode(weights)
    if prec == F32:
        return float(_L().or_gamma32(delta_value, chi_value, m, mode, wv, wl))
    return float(_L().or_gamma64(delta_value, chi_value, m, mode, wv, wl))


# ---------------------------------------------------------------- batches
def fused_topk(X, A, Qv, QA, k, weights=None, prec=F64, wildcard=None):
    """Exact top-k by (Gamma, id): returns ids [nq,k] int64, gamma [nq,k] f64, chi [nq,k].
    ``wildcard``: query code that leaves its position unconstrained (None: none)."""
    X, A, Qv, QA = _f32(X), _u8(A), _f32(Qv), _u8(QA)
    nq = Qv.shape[0]
    ids = np.empty((nq, k), np.int64)
    g = np.empty((nq, k), np.float64)
    ch = np.empty((nq, k), np.int32)
    mode, wv, wl = _mode(weights)
    _L().or_fused_topk(_p(X), _p(A), X.shape[0], X.shape[1], A.shape[1], _p(Qv), _p(QA), nq, k,
                       mode, wv, wl, prec, _p(ids), _p(g), _p(ch), _wild(wildcard))
    return ids, g, ch


def filtered_topk(X, A, Qv, QA, k, prec=F64, wildcard=None):
    """Hybrid ground truth G: k nearest by delta among exact attribute matches.
    Returns ids [nq,k] (-1 padded), delta [nq,k], |P| [nq]."""
    X, A, Qv, QA = _f32(X), _u8(A), _f32(Qv), _u8(QA)
    nq = Qv.shape[0]
    ids = np.empty((nq, k), np.int64)
    dl = np.empty((nq, k), np.float64)
    P = np.empty(nq, np.int64)
    _L().or_filtered_topk(_p(X), _p(A), X.shape[0], X.shape[1], A.shape[1], _p(Qv), _p(QA), nq,
                          k, prec, _p(ids), _p(dl), _p(P), _wild(wildcard))
    return ids, dl, P


def knn(X, A, K, weights=None, prec=F64, rows=None, vec_round=0):
    """Exact K nearest v != u by (Gamma, id) for every u (or the given rows).
    ``vec_round`` (ROUND_BF16 / ROUND_E4M3) computes them on the rounded rows."""
    X, A = _f32(X), _u8(A)
    if vec_round:
        X = round_rows(X, vec_round)
    N = X.shape[0]
    if rows is None:
        rp, nr = None, N
    else:
        rows = _i64(rows)
        rp, nr = _p(rows), rows.shape[0]
    ids = np.empty((nr, K), np.int64)
    g = np.empty((nr, K), np.float64)
    mode, wv, wl = _mode(weights)
    _L().or_knn(_p(X), _p(A), N, X.shape[1], A.shape[1], K, mode, wv, wl, prec, rp, nr, _p(ids),
                _p(g))
    return ids, g


def edge_select(X, A, cand, R, weights=None, prec=F64, rows=None):
    """Landing-zone edge selection over candidate lists cand [N,K] -> nbr [N,R] (-1 pad), deg [N].
    With ``rows`` (vertex ids), cand holds one row per listed vertex and so do the outputs."""
    X, A, cand = _f32(X), _u8(A), _i64(cand)
    nr, K = cand.shape
    if rows is None:
        rp = None
    else:
        rows = _i64(rows)
        assert rows.shape[0] == nr
        rp = _p(rows)
    nbr = np.empty((nr, R), np.int64)
    deg = np.empty(nr, np.int32)
    mode, wv, wl = _mode(weights)
    _L().or_edge_select(_p(X), _p(A), X.shape[0], X.shape[1], A.shape[1], _p(cand), K, R, mode,
                        wv, wl, prec, rp, nr, _p(nbr), _p(deg))
    return nbr, deg


def reverse_candidates(nbr, cap=64, rows=None):
    """Rows N(v) + up to ``cap`` smallest reverse sources {u : v in N(u)} -> [N, R+cap]
    (or one row per vertex listed in ``rows``)."""
    nbr = _i64(nbr)
    N, R = nbr.shape
    if rows is None:
        rp, nr = None, N
    else:
        rows = _i64(rows)
        rp, nr = _p(rows), rows.shape[0]
    out = np.empty((nr, R + cap), np.int64)
    _L().or_reverse_candidates(_p(nbr), N, R, cap, rp, nr, _p(out))
    return out


def build_graph(X, A, R=32, K=64, weights=None, prec=F32, reverse=True, rev_cap=64):
    """The whole composite-index build: C(u) = exact K nearest, landing-zone
    selection, then (reverse=True) the reverse-candidate second pass."""
    cand, _ = knn(X, A, K, weights=weights, prec=prec)
    nbr, deg = edge_select(X, A, cand, R, weights=weights, prec=prec)
    if reverse:
        nbr, deg = edge_select(X, A, reverse_candidates(nbr, rev_cap), R, weights=weights,
                               prec=prec)
    return nbr, deg, cand


def nsw_waves(N, wave_max):
    """Insertion waves [s, e) of the incremental build: vertex 0 alone, then waves of
    1, 2, 4, ... vertices, at most wave_max each."""
    waves, s = [], 1
    while s < N:
        e = min(N, s + min(s, wave_max))
        waves.append((s, e))
        s = e
    return waves


def nsw_seeds(v, s, seed, n=32):
    """Entry points of vertex v's insertion search in the graph of [0, s): min(n, s)
    consecutive ids (h + j) mod s from h = splitmix64(seed ^ mix64(v))[0] mod s, so every
    earlier vertex is a seed while s <= n; -1 pads the row."""
    h = splitmix64_stream(seed ^ mix64(v), 1)[0] % s
    row = [(h + j) % s for j in range(min(n, s))]
    return row + [-1] * (n - len(row))


def nsw_attribute_seeds(v, s, A, seed, n=32):
    """Attribute entry for vertex v's insertion search: P = the earlier vertices u < s whose
    attributes all equal v's, ascending; c = |P| > 0: min(n, c) of them evenly spaced,
    P[floor(j c / S)]; c = 0: the consecutive-id rule of nsw_seeds.  -1 pads the row."""
    P = np.nonzero((A[:s] == A[v]).all(axis=1))[0]
    c = len(P)
    if c == 0:
        return nsw_seeds(v, s, seed, n)
    S = min(n, c)
    row = [int(P[(j * c) // S]) for j in range(S)]
    return row + [-1] * (n - S)


def build_nsw(X, A, R=32, L=64, weights=None, seed=0, wave_max=4096, rev_cap=64, prec=F32,
              trace=False, entry=0):
    """Incremental build (NPG_nsw of Sec. 4.3, batched into insertion waves): the vertices
    of a wave [s, e) each search the graph of [0, s) (Alg. 2 with the nsw_seeds entry
    points, k = ef = L) for their candidates and keep a landing-zone selection of them
    (Def. 6); then every earlier vertex u that one of them selected re-selects its
    neighbours from N(u) plus those new sources (ascending ids, at most rev_cap).  Every
    wave sees the graph as it was when the wave began.  With trace=True also returns the
    candidate lists of every wave.  entry = 1 takes the entry points by attributes
    (nsw_attribute_seeds) instead of by id (nsw_seeds)."""
    X, A = _f32(X), _u8(A)
    N = X.shape[0]
    nbr = np.full((N, R), -1, np.int64)
    steps = []
    for s, e in nsw_waves(N, wave_max):
        W = np.arange(s, e)
        if entry == 1:
            seeds = np.array([nsw_attribute_seeds(int(v), s, A, seed) for v in W], np.int64)
        else:
            seeds = np.array([nsw_seeds(int(v), s, seed) for v in W], np.int64)
        r = search(X, A, nbr, X[W], A[W], L, L, seeds=seeds, weights=weights, prec=prec)
        cand = r["ids"]
        new_rows, _ = edge_select(X, A, cand, R, weights=weights, prec=prec, rows=W)
        if trace:
            steps.append((W, cand))
        sources = {}
        for i, v in enumerate(W):
            for u in new_rows[i]:
                if u >= 0:
                    sources.setdefault(int(u), []).append(int(v))
        nbr[W] = new_rows
        if sources:
            U = np.array(sorted(sources), np.int64)
            cu = np.full((len(U), R + rev_cap), -1, np.int64)
            for i, u in enumerate(U):
                row = [int(x) for x in nbr[u] if x >= 0] + sorted(sources[int(u)])[:rev_cap]
                cu[i, :len(row)] = row
            nbr[U], _ = edge_select(X, A, cu, R, weights=weights, prec=prec, rows=U)
    return (nbr, steps) if trace else nbr


def graph_quality(nbr, knn_ids) -> float:
    nbr, knn_ids = _i64(nbr), _i64(knn_ids)
    return float(_L().or_graph_quality(_p(nbr), nbr.shape[0], nbr.shape[1], _p(knn_ids),
                                       knn_ids.shape[1]))


SEED_RANDOM, SEED_ATTRIBUTE, SEED_GIVEN, SEED_ATTRIBUTE_NEAR = 0, 1, 2, 3


ROUND_NONE, ROUND_BF16, ROUND_E4M3, ROUND_F16 = 0, 1, 2, 3


def round_bf16(x) -> float:
    return float(_L().or_round_bf16(float(x)))


def round_e4m3(x) -> float:
    return float(_L().or_round_e4m3(float(x)))


def round_rows(X, mode):
    """A copy of X with every value rounded to bf16 (ROUND_BF16), fp8 e4m3 (ROUND_E4M3) or
    IEEE binary16 (ROUND_F16)."""
    Y = np.array(X, dtype=np.float32, order="C", copy=True)
    _L().or_round_rows(_p(Y), Y.size, int(mode))
    return Y


def search(X, A, nbr, Qv, QA, k, ef, h=1, seed=0, max_iters=1 << 30, weights=None, prec=F32,
           seed_mode=SEED_RANDOM, seeds=None, vec_round=ROUND_NONE, rerank=False,
           wildcard=None):
    """Serial Alg. 2 (+ two-stage routing when h > 1).  ``seed_mode`` picks the
    seed set B (random stream / attribute entry / the rows of ``seeds``, -1 =
    none).  ``vec_round`` scores candidates with X rounded to bf16 / fp8 e4m3;
    ``rerank`` re-scores the final pool with X itself before returning the first k.
    ``wildcard``: query code that leaves its position unconstrained; under the attribute
    seed modes such a query takes the mode's rule over the runs of its completions.
    Returns a dict with ids/gamma/chi [nq,k], ndc/expansions/status [nq]."""
    X, A, nbr, Qv, QA = _f32(X), _u8(A), _i64(nbr), _f32(Qv), _u8(QA)
    if seeds is not None:
        seeds = _i64(seeds)
        seed_mode = SEED_GIVEN
        sp, ns = _p(seeds), seeds.shape[1]
    else:
        sp, ns = None, 0
    nq = Qv.shape[0]
    ids = np.empty((nq, k), np.int64)
    g = np.empty((nq, k), np.float64)
    ch = np.empty((nq, k), np.int32)
    ndc = np.empty(nq, np.int64)
    ex = np.empty(nq, np.int64)
    st = np.empty(nq, np.int32)
    mode, wv, wl = _mode(weights)
    _L().or_search(_p(X), _p(A), X.shape[0], X.shape[1], A.shape[1], _p(nbr), nbr.shape[1],
                   _p(Qv), _p(QA), nq, k, ef, h, C.c_uint64(seed & (2**64 - 1)), max_iters,
                   mode, wv, wl, prec, seed_mode, sp, ns, int(vec_round), int(bool(rerank)),
                   _p(ids), _p(g), _p(ch), _p(ndc), _p(ex), _p(st), _wild(wildcard))
    return dict(ids=ids, gamma=g, chi=ch, ndc=ndc, expansions=ex, status=st)


# ---------------------------------------------------------------- entry cells
# Coarse cells for choosing where a search enters the graph (a project addition; the
# paper draws the seed set B of Alg. 2 at random): E centroids, the objects with ids
# floor(j N / E); every object belongs to the cell of its nearest centroid.
def cell_centroids(N, E):
    """Ids of the E centroid objects, floor(j N / E) for j < E."""
    return np.array([(j * N) // E for j in range(E)], np.int64)


def cells(X, E):
    """Cell of every object: the centroid j with the smallest (delta, j), delta by Eq. 1 in
    the canonical f32 form (the exact top-1 of the plain L2 brute force over the E
    centroid rows)."""
    X = _f32(X)
    cid = cell_centroids(X.shape[0], E)
    zeros = np.zeros((X.shape[0], 1), np.uint8)
    ids, _, _ = fused_topk(X[cid], zeros[:E], X, zeros, 1, weights=(1.0, 0.0), prec=F32)
    return ids[:, 0]


def nearest_cells(X, E, Qv, T):
    """The T cells whose centroids are nearest to each query by (delta, j), canonical f32."""
    X = _f32(X)
    cid = cell_centroids(X.shape[0], E)
    Qv = _f32(Qv)
    ids, _, _ = fused_topk(X[cid], np.zeros((E, 1), np.uint8), Qv,
                           np.zeros((Qv.shape[0], 1), np.uint8), T, weights=(1.0, 0.0), prec=F32)
    return ids


def cell_seeds(A, QA, cell_of, chosen, ef, seed=0):
    """Seed rows [nq, 32] (-1 padded) of the cell entry rule for closed queries: P = the
    objects whose attributes all equal the query's (ascending ids), S = min(ef, 32, |P|);
    B = the first S members of P in the chosen cells (chosen[q][0] first, ascending ids
    within a cell), then, while fewer than S, the evenly spaced members P[floor(j |P| / S2)]
    for j < S2 = S - |B| (repeats allowed; Alg. 2 evaluates an id once); |P| = 0: the
    first min(ef, 32) distinct ids of splitmix64(seed ^ mix64(q)) mod N (<= 64 draws)."""
    A, QA = np.asarray(A), np.asarray(QA)
    N = A.shape[0]
    out = np.full((QA.shape[0], 32), -1, np.int64)
    for q in range(QA.shape[0]):
        P = np.flatnonzero((A == QA[q]).all(axis=1))
        c = P.size
        if c == 0:
            want, row = min(ef, 32), []
            for x in splitmix64_stream(seed ^ mix64(q), 64):
                v = x % N
                if v not in row:
                    row.append(v)
                if len(row) == want:
                    break
        else:
            S = min(ef, 32, c)
            row = []
            for cell in chosen[q]:
                row += [int(v) for v in P[cell_of[P] == cell]]
            row = row[:S]
            S2 = S - len(row)
            row += [int(P[(j * c) // S2]) for j in range(S2)]
        out[q, :len(row)] = row
    return out


# ---------------------------------------------------------------- metrics
def recall(found, truth) -> float:
    """Eq. 3: mean over queries of |D & G| / k."""
    found, truth = np.asarray(found), np.asarray(truth)
    k = truth.shape[1]
    hits = [len(set(f[f >= 0].tolist()) & set(t[t >= 0].tolist())) for f, t in zip(found, truth)]
    return float(np.mean(hits) / k) if len(hits) else 0.0


def hybrid_recall(found, A, QA, truth, P):
    """Recall of Sec. 6.1: only returned ids whose attributes equal the query's
    count; the denominator is min(k, |P|); queries with |P| = 0 are excluded.
    Returns (recall, n_excluded)."""
    found, truth, A, QA = np.asarray(found), np.asarray(truth), np.asarray(A), np.asarray(QA)
    k = truth.shape[1]
    vals, excl = [], 0
    for f, t, qa, p in zip(found, truth, QA, P):
        if p == 0:
            excl += 1
            continue
        f = f[f >= 0]
        f = f[(A[f] == qa).all(axis=1)]
        vals.append(len(set(f.tolist()) & set(t[t >= 0].tolist())) / min(k, int(p)))
    return (float(np.mean(vals)) if vals else 0.0), excl
