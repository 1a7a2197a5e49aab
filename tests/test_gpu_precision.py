"""Distance error of the reduced-precision scoring copies against the fp64 oracle, on a
GIST-shaped set (d = 960, unit-normalised rows, m = 4 uniform attributes): for every
returned record of a bf16 or fp8-e4m3 search, with and without the f32 re-rank, the
reported Gamma is compared with the fp64 Gamma of the same object.

Bounds (curve iv, Gamma = delta (1 + chi/m)): a copy x~ of a row x moves delta by at
most ||x~ - x||_2 (triangle inequality).  bf16 rounds each component to 8 significant
bits: |x~_i - x_i| <= 2^-9 |x_i|, so ||x~ - x|| <= 2^-9 ||x||.  e4m3 keeps 4 significant
bits down to 2^-6 and a spacing of 2^-9 below it: |x~_i - x_i| <= 2^-4 |x_i| + 2^-10, so
||x~ - x|| <= 2^-4 ||x|| + 2^-10 sqrt(d).  The re-rank re-scores with the f32 rows, so
its values meet the f32 bound (1e-5 relative)."""
import math

import numpy as np
import pytest

import oracle as O
import synth
from helpers import dev, empty_out, ids_i64

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
def gist(nhq):
    w = synth.c3(N=100_000, nq=500)
    ix = nhq.Index.build(dev(w.X), dev(w.A), degree=32, K=64, knn_dtype=1)
    yield w, ix
    ix.close()


CASES = [("f32", 0, 0), ("bf16", 1, 0), ("bf16+rerank", 1, 1), ("fp8", 2, 0),
         ("fp8+rerank", 2, 1)]


@pytest.mark.parametrize("name,vec,rerank", CASES)
def test_distance_error_against_fp64(nhq, gist, name, vec, rerank):
    w, ix = gist
    ids, g, chi = empty_out(w.nq, 10)
    nhq.nhq_search(ix.handle, dev(w.Qv), dev(w.QA), 10, 64, ids, g, chi, seed=9, vec_dtype=vec,
                   rerank=rerank, seed_mode=nhq.SEED_ATTRIBUTE)
    torch.cuda.synchronize()
    got, gg, cc = ids_i64(ids), g.cpu().numpy().astype(np.float64), chi.cpu().numpy()
    norm = np.linalg.norm(w.X.astype(np.float64), axis=1)
    rel = []
    for q in range(w.nq):
        for j in range(10):
            i = got[q, j]
            if i < 0:
                continue
            g64 = O.gamma(O.delta(w.Qv[q], w.X[i], O.F64), O.chi(w.QA[q], w.A[i]), w.m)
            assert int(cc[q, j]) == O.chi(w.QA[q], w.A[i])
            if vec == 0 or rerank:
                tol = 1e-5 * g64
            elif vec == 1:
                tol = (1 + cc[q, j] / w.m) * 2.0 ** -9 * norm[i] + 1e-5 * g64
            else:
                tol = ((1 + cc[q, j] / w.m) * (2.0 ** -4 * norm[i] + 2.0 ** -10 * math.sqrt(w.d))
                       + 1e-5 * g64)
            assert abs(gg[q, j] - g64) <= tol, (name, q, j, gg[q, j], g64)
            rel.append(abs(gg[q, j] - g64) / g64 if g64 > 0 else 0.0)
    rel = np.array(rel)
    print(f"{name}: relative Gamma error vs fp64 over {rel.size} records: "
          f"max {rel.max():.3e}, mean {rel.mean():.3e}")
