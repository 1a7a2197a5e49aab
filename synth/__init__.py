"""Seeded synthetic inputs shaped like the paper's hybrid-query workloads.

This module is shared by the CUDA path's tests/bench and by the oracle's tests.
It holds no arithmetic of the method itself (no distance, no fusion, no search):
only random vectors, ordinally encoded attributes (Sec. 3.2, "ordinal encoding")
and query tuples.

The paper's datasets (SIFT1M, GIST1M, ...; Sec. 6.1, Tab. 2) are not available,
so each workload below stands in for one of them with its shape:

* ``c1``  small Gaussian mixture, N=10k, d=128, m=3 (cards 3/5/10 uniform).
* ``c2``  SIFT1M-shaped: N=1M, d=128, integer components 0..255 stored as f32,
          1,000 centroids; m=3 (cards 3/10/20, Zipf s=1).
* ``c3``  GIST1M-shaped: N=1M, d=960 unit-normalised rows; m=4 (2/5/10/50).
* ``c4``  N=1M, d=96, attributes correlated with the cluster (cards 5/20/100),
          query selectivity log-uniform in [1e-4, 1/3], mixed k and ef.
* ``c5``  N=10M, d=96 stored as f16, 4,096 centroids; m=3 (10/50/200 Zipf).

Every generator is a pure function of its arguments (seed = 1000 + config index
by default; queries come from an independent stream of the same seed).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload",
    "c1",
    "c2",
    "c3",
    "c4",
    "c5",
    "int_valued",
    "c5_queries",
    "gaussian_mixture",
    "zipf_attributes",
    "uniform_attributes",
    "mixed_k_ef",
]


@dataclass
class Workload:
    """One synthetic object set plus a query batch (Def. 1 and Def. 4)."""

    name: str
    X: np.ndarray  # [N, d] float32 feature vectors nu(e)
    A: np.ndarray  # [N, m] uint8 ordinal attribute codes l(e)
    Qv: np.ndarray  # [nq, d] float32 query vectors
    QA: np.ndarray  # [nq, m] uint8 query attribute tuples
    cards: tuple
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    @property
    def d(self) -> int:
        return int(self.X.shape[1])

    @property
    def m(self) -> int:
        return int(self.A.shape[1])

    @property
    def nq(self) -> int:
        return int(self.Qv.shape[0])


def _rngs(seed: int):
    ss = np.random.SeedSequence(seed)
    base, query, attr, qattr = ss.spawn(4)
    return (np.random.default_rng(base), np.random.default_rng(query),
            np.random.default_rng(attr), np.random.default_rng(qattr))


def gaussian_mixture(rng, n, centroids, sigma, chunk=1 << 16):
    """Points = centroid[c] + N(0, sigma^2 I), component c uniform. Returns (X, comp)."""
    k, d = centroids.shape
    comp = rng.integers(0, k, size=n)
    X = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        noise = rng.standard_normal((e - s, d), dtype=np.float32)
        X[s:e] = centroids[comp[s:e]] + np.float32(sigma) * noise
    return X, comp


def uniform_attributes(rng, n, cards):
    A = np.empty((n, len(cards)), dtype=np.uint8)
    for i, c in enumerate(cards):
        A[:, i] = rng.integers(0, c, size=n)
    return A


def _zipf_probs(card, s=1.0):
    w = 1.0 / np.power(np.arange(1, card + 1, dtype=np.float64), s)
    return w / w.sum()


def zipf_attributes(rng, n, cards, s=1.0):
    """Attribute value v of a card-ary attribute drawn with P(v) ~ 1/(v+1)^s."""
    A = np.empty((n, len(cards)), dtype=np.uint8)
    for i, c in enumerate(cards):
        A[:, i] = rng.choice(c, size=n, p=_zipf_probs(c, s))
    return A


def _check_cards(cards):
    if not 1 <= len(cards) <= 32 or any(c < 1 or c > 256 for c in cards):
        raise ValueError("1..32 attributes with cardinality 1..256 are supported")


def c1(N=10_000, nq=1_000, d=128, cards=(3, 5, 10), n_comp=100, seed=1000):
    """Small plain case: 100-component Gaussian mixture, uniform attributes."""
    _check_cards(cards)
    rb, rq, ra, rqa = _rngs(seed)
    cent = rb.standard_normal((n_comp, d), dtype=np.float32)
    X, _ = gaussian_mixture(rb, N, cent, 0.1)
    Qv, _ = gaussian_mixture(rq, nq, cent, 0.1)
    A = uniform_attributes(ra, N, cards)
    QA = uniform_attributes(rqa, nq, cards)
    return Workload("c1", X, A, Qv, QA, tuple(cards),
                    dict(seed=seed, n_comp=n_comp, dist="gaussian-mixture sigma=0.1"))


def _int_mixture(rng, n, cent, sigma, chunk=1 << 16):
    k, d = cent.shape
    comp = rng.integers(0, k, size=n)
    X = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        v = cent[comp[s:e]] + np.float32(sigma) * rng.standard_normal((e - s, d), dtype=np.float32)
        X[s:e] = np.clip(np.rint(v), 0, 255)
    return X, comp


def c2(N=1_000_000, nq=10_000, d=128, cards=(3, 10, 20), n_comp=1_000, seed=1001,
       query_stream=0):
    """SIFT1M-shaped: integer-valued components 0..255 stored as f32, Zipf attributes.

    With integer components the squared distance is an integer <= d*255^2, which
    for d <= 256 is below 2^24, so it is exact in f32 in any summation order.
    query_stream > 0 draws the queries from another independent stream (same
    object set, same mixture): e.g. training queries for the learned stop.
    """
    _check_cards(cards)
    rb, rq, ra, rqa = _rngs(seed)
    if query_stream:
        rq, rqa = (np.random.default_rng(x)
                   for x in np.random.SeedSequence([seed, query_stream]).spawn(2))
    cent = np.clip(np.rint(64.0 + 40.0 * rb.standard_normal((n_comp, d))), 0, 255).astype(np.float32)
    X, _ = _int_mixture(rb, N, cent, 20.0)
    Qv, _ = _int_mixture(rq, nq, cent, 20.0)
    A = zipf_attributes(ra, N, cards)
    QA = zipf_attributes(rqa, nq, cards)
    return Workload("c2", X, A, Qv, QA, tuple(cards),
                    dict(seed=seed, n_comp=n_comp, dist="integer mixture 0..255, sigma=20"))


def int_valued(N, nq, d, cards=(3, 10, 20), n_comp=16, seed=7, zipf=True):
    """Small integer-valued workload (same recipe as ``c2``) for exact parity tests."""
    w = c2(N=N, nq=nq, d=d, cards=cards, n_comp=n_comp, seed=seed)
    if not zipf:
        _, _, ra, rqa = _rngs(seed)
        w.A = uniform_attributes(ra, N, cards)
        w.QA = uniform_attributes(rqa, nq, cards)
    w.name = f"int{N}x{d}"
    return w


def c3(N=1_000_000, nq=10_000, d=960, cards=(2, 5, 10, 50), n_comp=1_000, seed=1002,
       query_stream=0):
    """GIST1M-shaped: unit-normalised Gaussian-mixture rows, 4 uniform attributes.
    query_stream > 0 draws the queries from another independent stream (as in c2)."""
    _check_cards(cards)
    rb, rq, ra, rqa = _rngs(seed)
    if query_stream:
        rq, rqa = (np.random.default_rng(x)
                   for x in np.random.SeedSequence([seed, query_stream]).spawn(2))
    cent = rb.standard_normal((n_comp, d), dtype=np.float32)
    X, _ = gaussian_mixture(rb, N, cent, 0.5)
    Qv, _ = gaussian_mixture(rq, nq, cent, 0.5)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    Qv /= np.linalg.norm(Qv, axis=1, keepdims=True)
    A = uniform_attributes(ra, N, cards)
    QA = uniform_attributes(rqa, nq, cards)
    return Workload("c3", X, A, Qv, QA, tuple(cards), dict(seed=seed, n_comp=n_comp))


def c4(N=1_000_000, nq=100_000, d=96, cards=(5, 20, 100), n_comp=1_000, seed=1003,
       sel_lo=1e-4, sel_hi=1.0 / 3.0):
    """Attributes correlated with the cluster; query selectivity log-uniform.

    Each attribute value is drawn from a Zipf preference (s = 3): with probability
    1/4 the object's centroid relabels it (each centroid has its own random
    relabelling, the correlation), otherwise one global labelling applies (so
    frequent tuples exist across clusters, up to a selectivity near 1/3).  Query tuples are picked among the
    tuples that occur in the base set so that |P|/N is close to a log-uniform
    target in [sel_lo, sel_hi].
    """
    _check_cards(cards)
    rb, rq, ra, rqa = _rngs(seed)
    cent = rb.standard_normal((n_comp, d), dtype=np.float32)
    X, comp = gaussian_mixture(rb, N, cent, 0.3)
    Qv, _ = gaussian_mixture(rq, nq, cent, 0.3)
    A = np.empty((N, len(cards)), dtype=np.uint8)
    for i, c in enumerate(cards):
        perms = np.argsort(ra.random((n_comp, c)), axis=1).astype(np.uint8)
        draw = ra.choice(c, size=N, p=_zipf_probs(c, 3.0))
        local = ra.random(N) < 0.25
        A[:, i] = np.where(local, perms[comp, draw], draw).astype(np.uint8)
    # tuple frequencies
    mult = np.cumprod((1,) + tuple(cards[:-1]))
    code = (A.astype(np.int64) * mult).sum(axis=1)
    uniq, counts = np.unique(code, return_counts=True)
    sel = counts / N
    order = np.argsort(sel)
    target = np.exp(rqa.uniform(np.log(sel_lo), np.log(sel_hi), size=nq))
    pos = np.clip(np.searchsorted(sel[order], target), 0, len(order) - 1)
    chosen = uniq[order[pos]]
    QA = np.empty((nq, len(cards)), dtype=np.uint8)
    rem = chosen.copy()
    for i, c in enumerate(cards):
        QA[:, i] = rem % c
        rem //= c
    return Workload("c4", X, A, Qv, QA, tuple(cards), dict(seed=seed, n_comp=n_comp))


def c5_queries(nq, query_stream, d=96, cards=(10, 50, 200), n_comp=4_096, seed=1004):
    """Queries of the c5 mixture from an independent query stream, without generating the
    10M-object base set (the centroids are the base stream's first draw): training
    queries for the learned parts.  Returns (Qv, QA)."""
    _check_cards(cards)
    rb, _, _, _ = _rngs(seed)
    rq, rqa = (np.random.default_rng(x)
               for x in np.random.SeedSequence([seed, query_stream]).spawn(2))
    cent = rb.standard_normal((n_comp, d), dtype=np.float32)
    Qv, _ = gaussian_mixture(rq, nq, cent, 0.3)
    Qv = Qv.astype(np.float16).astype(np.float32)
    return Qv, zipf_attributes(rqa, nq, cards)


def c5(N=10_000_000, nq=50_000, d=96, cards=(10, 50, 200), n_comp=4_096, seed=1004):
    """Largest case: Gaussian mixture stored as f16 (returned here as f32 values
    that are exactly representable in f16), Zipf attributes."""
    _check_cards(cards)
    rb, rq, ra, rqa = _rngs(seed)
    cent = rb.standard_normal((n_comp, d), dtype=np.float32)
    X, _ = gaussian_mixture(rb, N, cent, 0.3)
    Qv, _ = gaussian_mixture(rq, nq, cent, 0.3)
    X = X.astype(np.float16).astype(np.float32)
    Qv = Qv.astype(np.float16).astype(np.float32)
    A = zipf_attributes(ra, N, cards)
    QA = zipf_attributes(rqa, nq, cards)
    return Workload("c5", X, A, Qv, QA, tuple(cards), dict(seed=seed, n_comp=n_comp))


def mixed_k_ef(nq, seed=2003, ks=(1, 10, 100), ef_lo=16, ef_hi=512):
    """Per-query k drawn from ``ks`` and ef uniform in [max(ef_lo, k), ef_hi]."""
    r = np.random.default_rng(seed)
    k = r.choice(np.asarray(ks, dtype=np.int32), size=nq)
    lo = np.maximum(k, ef_lo)
    ef = (lo + np.floor(r.random(nq) * (ef_hi - lo + 1))).astype(np.int32)
    return k.astype(np.int32), ef
