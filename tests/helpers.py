"""Shared helpers for the GPU tests: device placement, id conversion, and the
near-tie-aware comparison used where float summation order may differ."""
import numpy as np

NONE = 0xFFFFFFFF


def dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def to_u32_graph(nbr):
    nbr = np.asarray(nbr)
    return np.where(nbr < 0, NONE, nbr).astype(np.uint32)


def ids_i64(t):
    """GPU u32 ids (0xFFFFFFFF = none) -> int64 with -1 = none."""
    a = t.cpu().numpy().astype(np.int64) if hasattr(t, "cpu") else np.asarray(t, np.int64)
    a[a == NONE] = -1
    return a


def empty_out(Q, k, device="cuda:0"):
    import torch

    return (torch.empty((Q, k), dtype=torch.uint32, device=device),
            torch.empty((Q, k), dtype=torch.float32, device=device),
            torch.empty((Q, k), dtype=torch.uint8, device=device))


def gamma64_of(O, X, A, qv, qa, ids, weights):
    """f64 Gamma of the given objects against one query (oracle arithmetic)."""
    out = []
    for i in ids:
        if i < 0:
            out.append(np.inf)
            continue
        out.append(O.gamma(O.delta(qv, X[i], O.F64), O.chi(qa, A[i]), A.shape[1], weights, O.F64))
    return np.array(out)


def assert_topk_near_tie_equal(O, X, A, Qv, QA, got_ids, got_g, ref_ids, ref_g, weights,
                               rtol=1e-5):
    """Values within rtol of the f64 oracle; ids equal except at near-ties, where the
    f64 Gamma of both ids must agree within rtol.  Returns the number of near-tie swaps."""
    swaps = 0
    for q in range(got_ids.shape[0]):
        assert np.allclose(got_g[q], ref_g[q], rtol=rtol, atol=0), q
        if (got_ids[q] == ref_ids[q]).all():
            continue
        g_got = gamma64_of(O, X, A, Qv[q], QA[q], got_ids[q], weights)
        g_ref = gamma64_of(O, X, A, Qv[q], QA[q], ref_ids[q], weights)
        assert np.allclose(g_got, g_ref, rtol=rtol, atol=0), q
        assert len(set(got_ids[q].tolist())) == len(got_ids[q])
        swaps += int((got_ids[q] != ref_ids[q]).sum())
    return swaps
