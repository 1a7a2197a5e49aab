"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol declared in include/*.h, and rejects bad arguments before any CUDA work."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2203_13601_gb300 import build as B

    B.build()
    import paper_2203_13601_gb300 as nhq

    return nhq.load_library()


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(nhq_[a-z_0-9]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("nhq_build", "nhq_search", "nhq_search_batched", "nhq_brute_force",
                     "nhq_knn", "nhq_edge_select", "nhq_save", "nhq_load", "nhq_free"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_mirrors_the_abi():
    import paper_2203_13601_gb300 as nhq

    missing = [n for n in _declared_functions() if not hasattr(nhq, n)]
    assert not missing, missing


def test_version_and_empty_error(lib):
    import paper_2203_13601_gb300 as nhq

    assert nhq.nhq_version() == 1
    assert isinstance(nhq.nhq_last_error(), str)


def test_argument_errors_before_cuda(lib):
    import paper_2203_13601_gb300 as nhq

    out = C.c_void_p()
    w = nhq._Weights(0, 1.0, 0.0)
    x = np.zeros((4, 3), np.float32)
    a = np.zeros((4, 33), np.uint8)
    # m = 33 attributes is outside 1..32
    st = lib.nhq_index_create(x.ctypes.data, 4, 3, a.ctypes.data, 33, w, None, C.byref(out))
    assert st == nhq.ERR_ARG and out.value is None
    assert "m must be" in nhq.nhq_last_error()
    st = lib.nhq_index_create(x.ctypes.data, 4, 3, a.ctypes.data, 0, w, None, C.byref(out))
    assert st == nhq.ERR_ARG and out.value is None
    # N = 0
    st = lib.nhq_index_create(x.ctypes.data, 0, 3, a.ctypes.data, 2, w, None, C.byref(out))
    assert st == nhq.ERR_ARG
    # curve ii needs c >= 1 (its adjusted chi must grow with chi)
    st = lib.nhq_index_create(x.ctypes.data, 4, 3, a.ctypes.data, 2, nhq._Weights(3, 1.0, 0.5),
                              None, C.byref(out))
    assert st == nhq.ERR_ARG and "harmonic" in nhq.nhq_last_error()
    # negative constant weight
    st = lib.nhq_index_create(x.ctypes.data, 4, 3, a.ctypes.data, 2, nhq._Weights(1, -1.0, 1.0),
                              None, C.byref(out))
    assert st == nhq.ERR_ARG
    # NULL index everywhere
    p = nhq._SearchParams()
    assert lib.nhq_search(None, None, None, 1, 10, 10, C.byref(p), None, None, None, None, None,
                          None, None) == nhq.ERR_ARG
    assert lib.nhq_brute_force(None, None, None, 1, 10, None, None, None, None, None) == nhq.ERR_ARG
    assert lib.nhq_index_build(None, 32, None, None) == nhq.ERR_ARG
    assert lib.nhq_save(None, b"/tmp/x") == nhq.ERR_ARG
    lib.nhq_free(None)  # no-op
    # shard merge: counts checked before any CUDA work
    assert lib.nhq_merge_topk(0, 1, 1, 1, None, None, None, None, None, None, None,
                              None) == nhq.ERR_ARG
    assert "P must be" in nhq.nhq_last_error()
    assert lib.nhq_merge_topk(2, 1, 0, 1, None, None, None, None, None, None, None,
                              None) == nhq.ERR_ARG
    assert lib.nhq_merge_topk(2, 1, 4, 4, None, None, None, None, None, None, None,
                              None) == nhq.ERR_ARG
    assert lib.nhq_postfilter(1, 0, 1, None, None, None, None, None, None) == nhq.ERR_ARG
    assert lib.nhq_postfilter(1, 4, 2, None, None, None, None, None, None) == nhq.ERR_ARG
    # the wildcard switch takes 0 or 1
    assert lib.nhq_brute_force_wildcard(None, None, None, 1, 10, None, 2, None, None, None,
                                        None) == nhq.ERR_ARG
    assert "wildcard must be" in nhq.nhq_last_error()
    assert lib.nhq_brute_force_wildcard(None, None, None, 1, 10, None, 1, None, None, None,
                                        None) == nhq.ERR_ARG


def test_load_rejects_missing_and_corrupt_files(lib, tmp_path):
    import paper_2203_13601_gb300 as nhq

    out = C.c_void_p()
    assert lib.nhq_load(str(tmp_path / "absent.idx").encode(), None, C.byref(out)) == nhq.ERR_IO
    bad = tmp_path / "bad.idx"
    bad.write_bytes(b"NOTANIDX" + b"\0" * 64)
    assert lib.nhq_load(str(bad).encode(), None, C.byref(out)) == nhq.ERR_IO
    assert "not an index file" in nhq.nhq_last_error()
    # header {version, N, d, m, R, weight mode, 0, 0} and the two weights
    def header(version, m, widths=None, shifts=None):
        h = np.array([version, 10, 4, m, 0, 0, 0, 0], np.int32).tobytes()
        h += np.array([1.0, 0.0], np.float32).tobytes()
        if version == 2:
            sh = np.zeros(32, np.uint8) if shifts is None else np.asarray(shifts, np.uint8)
            wd = np.zeros(32, np.uint8) if widths is None else np.asarray(widths, np.uint8)
            h += sh.tobytes() + wd.tobytes()
        return b"NHQIDX01" + h
    cases = {
        "v3": header(3, 2),
        "v1 with 5 attributes": header(1, 5),
        "v2 with a zero-width field": header(2, 2, widths=[8] + [0] * 31,
                                             shifts=[0, 8] + [0] * 30),
        "v2 with a field past bit 31": header(2, 1, widths=[9] + [0] * 31,
                                              shifts=[30] + [0] * 31),
        "v2 with 33 attributes": header(2, 33),
    }
    for name, blob in cases.items():
        f = tmp_path / "h.idx"
        f.write_bytes(blob + b"\0" * 16)
        assert lib.nhq_load(str(f).encode(), None, C.byref(out)) == nhq.ERR_IO, name
        assert "not an index file" in nhq.nhq_last_error(), name
    # a valid version-2 header over a truncated body
    f = tmp_path / "t.idx"
    f.write_bytes(header(2, 2, widths=[8, 8] + [0] * 30, shifts=[0, 8] + [0] * 30) + b"\0" * 8)
    assert lib.nhq_load(str(f).encode(), None, C.byref(out)) == nhq.ERR_IO
    assert "truncated" in nhq.nhq_last_error()


def test_binding_type_checks():
    import paper_2203_13601_gb300 as nhq

    with pytest.raises(TypeError):
        nhq._ptr(np.zeros(3, np.float64), np.float32)
    with pytest.raises(ValueError):
        nhq._ptr(np.zeros((3, 4), np.float32).T, np.float32)
    with pytest.raises(ValueError):
        nhq._ptr(np.zeros((3, 4), np.float32), np.float32, (4, 3))
