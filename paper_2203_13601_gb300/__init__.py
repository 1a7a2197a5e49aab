"""GB300-native hybrid-query search (NHQ, arXiv 2203.13601) -- Python binding.

Every function below forwards to the C ABI of ``include/nhq.h`` with the same
name; this module only checks shapes/dtypes and passes pointers.  All compute
runs in the CUDA library ``_build/libnhq.so`` (built by ``build.py`` for
sm_103a).  Importing this module does not need a GPU; calling a function does
need the library, and a missing library raises ``RuntimeError``: there is no
CPU fallback.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; host arrays are
copied through the library's staging buffers and the call then synchronises.
``stream`` defaults to torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

__all__ = [
    "NHQError", "Index", "load_library", "library_path",
    "W_PROPORTIONAL", "W_CONSTANT", "W_FILTER", "W_HARMONIC", "VEC_F32", "VEC_BF16", "VEC_FP8E4M3",
    "VEC_F16", "F32", "F16", "BF16", "nhq_index_create_typed", "nhq_build_typed",
    "SEED_RANDOM", "SEED_ATTRIBUTE", "SEED_GIVEN", "SEED_ATTRIBUTE_NEAR",
    "nhq_last_error", "nhq_version", "nhq_index_create", "nhq_free", "nhq_index_info",
    "nhq_pack_attributes", "nhq_knn", "nhq_knn_bf16", "nhq_edge_select", "nhq_reverse_candidates",
    "nhq_index_set_graph", "nhq_index_get_graph", "nhq_index_build", "nhq_build",
    "nhq_brute_force", "nhq_brute_force_wildcard", "nhq_search", "nhq_search_batched", "nhq_save", "nhq_load",
    "nhq_brute_force_noalloc", "nhq_search_trace", "nhq_mlp_forward", "nhq_mlp_grad",
    "nhq_mlp_train", "MLP_INPUTS", "MLP_HIDDEN", "MLP_PARAMS", "nhq_autotune_search",
    "nhq_search_graph_create", "nhq_search_graph_launch", "nhq_search_graph_free",
    "nhq_merge_topk", "nhq_postfilter", "nhq_knn_nndescent", "nhq_index_build_nsw",
    "nhq_autotune_beam", "nhq_recall", "nhq_autotune", "nhq_autotune_batched",
    "nhq_search_graph_create_batched", "SEED_CELL_NEAREST", "SEED_CELL_LEARNED",
    "ENTRY_HIDDEN", "nhq_index_build_cells", "nhq_index_cells", "nhq_entry_param_count",
    "nhq_entry_forward", "nhq_entry_grad", "nhq_entry_train", "nhq_entry_labels",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libnhq.so")

W_PROPORTIONAL, W_CONSTANT, W_FILTER, W_HARMONIC = 0, 1, 2, 3
VEC_F32, VEC_BF16, VEC_FP8E4M3, VEC_F16 = 0, 1, 2, 3
F32, F16, BF16 = 0, 1, 2  # nhq_dtype of the input vectors
SEED_RANDOM, SEED_ATTRIBUTE, SEED_GIVEN, SEED_ATTRIBUTE_NEAR = 0, 1, 2, 3
SEED_CELL_NEAREST, SEED_CELL_LEARNED = 4, 5
ENTRY_HIDDEN = 64
MLP_INPUTS, MLP_HIDDEN = 8, 64
MLP_PARAMS = MLP_INPUTS * MLP_HIDDEN + 2 * MLP_HIDDEN + 1
OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_ITER_LIMIT, ERR_IO = range(6)
NONE_ID = 0xFFFFFFFF


class NHQError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"nhq status {status}: {message}")
        self.status = status


class _Weights(C.Structure):
    _fields_ = [("mode", C.c_int32), ("w_v", C.c_float), ("w_l", C.c_float)]


class _BuildParams(C.Structure):
    _fields_ = [("K", C.c_int32), ("reverse", C.c_int32), ("reverse_cap", C.c_int32),
                ("knn_dtype", C.c_int32)]


class _SearchParams(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("h", C.c_int32), ("max_iters", C.c_int32),
                ("warps_per_block", C.c_int32), ("hash_bits", C.c_int32),
                ("vec_dtype", C.c_int32), ("rerank", C.c_int32), ("seed_mode", C.c_int32),
                ("n_seeds", C.c_int32), ("seeds", C.c_void_p), ("stop_model", C.c_void_p),
                ("stop_threshold", C.c_float), ("stop_min", C.c_int32),
                ("stop_every", C.c_int32), ("wildcard", C.c_int32),
                ("warps_per_query", C.c_int32), ("entry_model", C.c_void_p),
                ("entry_cells", C.c_int32), ("cells_out", C.c_void_p),
                ("tile_rows", C.c_int32)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _LIB_PATH


def load_library():
    """Load libnhq.so (build it first with ``build.build()``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: run paper_2203_13601_gb300.build.build()"
                               " (the CUDA library is required; there is no CPU fallback)")
        lib = C.CDLL(_LIB_PATH)
        P, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        S = C.c_int  # nhq_status
        sig = {
            "nhq_last_error": (C.c_char_p, []),
            "nhq_version": (i32, []),
            "nhq_index_create": (S, [P, i64, i32, P, i32, _Weights, P, C.POINTER(P)]),
            "nhq_index_create_typed": (S, [P, i32, i64, i32, P, i32, _Weights, P, C.POINTER(P)]),
            "nhq_build_typed": (S, [P, i32, i64, i32, P, i32, i32, _Weights,
                                    C.POINTER(_BuildParams), P, C.POINTER(P)]),
            "nhq_free": (None, [P]),
            "nhq_index_info": (S, [P, P, P, P, P]),
            "nhq_pack_attributes": (S, [P, i64, i32, P, P]),
            "nhq_knn": (S, [P, i32, P, P, P]),
            "nhq_knn_bf16": (S, [P, i32, P, P, P]),
            "nhq_knn_nndescent": (S, [P, i32, i32, C.c_uint64, P, P, P, P]),
            "nhq_index_build_nsw": (S, [P, i32, i32, i32, i32, i32, C.c_uint64, P]),
            "nhq_edge_select": (S, [P, P, i32, i32, P, P]),
            "nhq_reverse_candidates": (S, [P, P, i32, i32, P, P]),
            "nhq_index_set_graph": (S, [P, P, i32, P]),
            "nhq_index_get_graph": (S, [P, P, P]),
            "nhq_index_build": (S, [P, i32, C.POINTER(_BuildParams), P]),
            "nhq_build": (S, [P, i64, i32, P, i32, i32, _Weights, C.POINTER(_BuildParams), P,
                              C.POINTER(P)]),
            "nhq_brute_force": (S, [P, P, P, i64, i32, C.POINTER(_Weights), P, P, P, P]),
            "nhq_brute_force_wildcard": (S, [P, P, P, i64, i32, C.POINTER(_Weights), i32, P, P,
                                             P, P]),
            "nhq_merge_topk": (S, [i32, i64, i32, i32, P, P, P, P, P, P, P, P]),
            "nhq_postfilter": (S, [i64, i32, i32, P, P, P, P, P, P]),
            "nhq_search": (S, [P, P, P, i64, i32, i32, C.POINTER(_SearchParams), P, P, P, P, P,
                               P, P]),
            "nhq_search_batched": (S, [P, P, P, i64, P, P, i32, C.POINTER(_SearchParams), P, P, P,
                                       P, P, P, P]),
            "nhq_brute_force_noalloc": (S, [P, P, i64, i32, i32, P, P, i64, i32, _Weights, P, P,
                                            P, P]),
            "nhq_autotune_search": (S, [P, P, P, i64, i32, i32, C.POINTER(_SearchParams), P,
                                        C.POINTER(C.c_float), P]),
            "nhq_autotune_beam": (S, [P, P, P, i64, i32, P, i32, P, C.c_float,
                                      C.POINTER(_SearchParams), P, C.POINTER(i32),
                                      C.POINTER(C.c_float), C.POINTER(C.c_float), P]),
            "nhq_recall": (S, [P, i32, P, i32, i64, C.POINTER(C.c_float), P]),
            "nhq_index_build_cells": (S, [P, i32, P]),
            "nhq_index_cells": (S, [P, C.POINTER(i32), P, P]),
            "nhq_entry_param_count": (i64, [i32, i32]),
            "nhq_entry_forward": (S, [P, i32, i32, P, i64, P, P]),
            "nhq_entry_grad": (S, [P, i32, i32, P, P, i64, P, P, P]),
            "nhq_entry_train": (S, [P, i32, i32, P, P, i64, i32, i32, C.c_float, P]),
            "nhq_entry_labels": (S, [P, P, i32, i64, P, P]),
            "nhq_search_graph_create": (S, [P, P, P, i64, i32, i32, C.POINTER(_SearchParams), P,
                                            P, P, C.POINTER(P)]),
            "nhq_search_graph_create_batched": (S, [P, P, P, i64, P, P, i32,
                                                    C.POINTER(_SearchParams), P, P, P,
                                                    C.POINTER(P)]),
            "nhq_autotune_batched": (S, [P, P, P, i64, P, P, i32, C.POINTER(_SearchParams), P,
                                         C.POINTER(C.c_float), P]),
            "nhq_search_graph_launch": (S, [P, P]),
            "nhq_search_graph_free": (None, [P]),
            "nhq_search_trace": (S, [P, P, P, i64, i32, i32, C.POINTER(_SearchParams), P, P, P,
                                     i64, C.POINTER(C.c_int64), P]),
            "nhq_mlp_forward": (S, [P, P, i64, P, P]),
            "nhq_mlp_grad": (S, [P, P, P, i64, P, P, P]),
            "nhq_mlp_train": (S, [P, P, P, i64, i32, i32, C.c_float, P]),
            "nhq_save": (S, [P, C.c_char_p]),
            "nhq_load": (S, [C.c_char_p, P, C.POINTER(P)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


# ------------------------------------------------------------------ marshalling
def _ptr(a, dtype, shape=None, name="array"):
    """Data pointer of a contiguous torch tensor / numpy array with the given dtype."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(dtype):
            raise TypeError(f"{name}: dtype {a.dtype}, expected {np.dtype(dtype)}")
        if not a.flags.c_contiguous:
            raise ValueError(f"{name} must be C-contiguous")
        shp = a.shape
        p = a.ctypes.data
    else:  # torch tensor
        import torch

        want = {np.float32: torch.float32, np.uint8: torch.uint8, np.int32: torch.int32,
                np.uint32: torch.uint32}[dtype]
        if a.dtype != want:
            raise TypeError(f"{name}: dtype {a.dtype}, expected {want}")
        if not a.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        shp = tuple(a.shape)
        p = a.data_ptr()
    if shape is not None and tuple(shp) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(shp)}, expected {tuple(shape)}")
    return p


def _shape(a):
    return tuple(a.shape)


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


def _weights(weights):
    if weights is None or weights == "proportional":
        return _Weights(W_PROPORTIONAL, 1.0, 0.0)
    if weights == "filter":
        return _Weights(W_FILTER, 1.0, 0.0)
    if weights == "harmonic":  # curve i of Sec. 6.5
        return _Weights(W_HARMONIC, 1.0, 0.0)
    if weights[0] == "harmonic":  # curve ii with constant c
        return _Weights(W_HARMONIC, 1.0, float(weights[1]))
    wv, wl = weights
    return _Weights(W_CONSTANT, float(wv), float(wl))


def _check(status):
    if status != OK:
        raise NHQError(status, load_library().nhq_last_error().decode())


# ------------------------------------------------------------------ ABI mirror
def nhq_last_error() -> str:
    return load_library().nhq_last_error().decode()


def nhq_version() -> int:
    return int(load_library().nhq_version())


def _vec_dtype_of(vectors):
    """nhq_dtype and element type of an input array (f32, f16 or bf16)."""
    name = str(vectors.dtype).replace("torch.", "")
    if name == "float16":
        return F16, np.float16
    if name == "bfloat16":
        return BF16, "bfloat16"
    return F32, np.float32


def _vec_ptr(vectors, N, d):
    dt, _ = _vec_dtype_of(vectors)
    if dt == F32:
        return dt, _ptr(vectors, np.float32, (N, d), "vectors")
    if tuple(vectors.shape) != (N, d) or not (vectors.is_contiguous() if hasattr(
            vectors, "is_contiguous") else vectors.flags.c_contiguous):
        raise ValueError("vectors must be a contiguous [N, d] array")
    return dt, vectors.data_ptr() if hasattr(vectors, "data_ptr") else vectors.ctypes.data


def nhq_index_create(vectors, attributes, weights=None, stream=None) -> int:
    N, d = _shape(vectors)
    m = _shape(attributes)[1]
    out = C.c_void_p()
    _check(load_library().nhq_index_create(_ptr(vectors, np.float32, (N, d), "vectors"), N, d,
                                           _ptr(attributes, np.uint8, (N, m), "attributes"), m,
                                           _weights(weights), _stream(stream), C.byref(out)))
    return out.value


def nhq_index_create_typed(vectors, attributes, weights=None, stream=None) -> int:
    """nhq_index_create for f32, f16 or bf16 vectors (the type is taken from the array)."""
    N, d = _shape(vectors)
    m = _shape(attributes)[1]
    dt, vp = _vec_ptr(vectors, N, d)
    out = C.c_void_p()
    _check(load_library().nhq_index_create_typed(vp, dt, N, d,
                                                 _ptr(attributes, np.uint8, (N, m), "attributes"),
                                                 m, _weights(weights), _stream(stream),
                                                 C.byref(out)))
    return out.value


def nhq_free(index) -> None:
    if index:
        load_library().nhq_free(index)


def nhq_index_info(index):
    N, d, m, R = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(load_library().nhq_index_info(index, C.byref(N), C.byref(d), C.byref(m), C.byref(R)))
    return N.value, d.value, m.value, R.value


def nhq_pack_attributes(attributes, packed, stream=None) -> None:
    n, m = _shape(attributes)
    _check(load_library().nhq_pack_attributes(_ptr(attributes, np.uint8, (n, m), "attributes"),
                                              n, m, _ptr(packed, np.uint32, (n,), "packed"),
                                              _stream(stream)))


def nhq_knn(index, K, cand_ids, cand_dist=None, stream=None) -> None:
    N = nhq_index_info(index)[0]
    _check(load_library().nhq_knn(index, K, _ptr(cand_ids, np.uint32, (N, K), "cand_ids"),
                                  _ptr(cand_dist, np.float32, (N, K), "cand_dist"),
                                  _stream(stream)))


def nhq_knn_bf16(index, K, cand_ids, cand_dist=None, stream=None) -> None:
    N = nhq_index_info(index)[0]
    _check(load_library().nhq_knn_bf16(index, K, _ptr(cand_ids, np.uint32, (N, K), "cand_ids"),
                                       _ptr(cand_dist, np.float32, (N, K), "cand_dist"),
                                       _stream(stream)))


def nhq_knn_nndescent(index, K, cand_ids, cand_dist=None, max_iters=12, seed=0x2203,
                      stream=None) -> int:
    """Candidate sets by NN-descent into cand_ids [N, K] (and cand_dist); returns the
    number of iterations run."""
    N = nhq_index_info(index)[0]
    it = C.c_int32(0)
    _check(load_library().nhq_knn_nndescent(
        index, K, max_iters, C.c_uint64(int(seed) & (2**64 - 1)),
        _ptr(cand_ids, np.uint32, (N, K), "cand_ids"),
        _ptr(cand_dist, np.float32, (N, K), "cand_dist"), C.byref(it), _stream(stream)))
    return it.value


def nhq_index_build_nsw(index, degree, L=64, wave_max=4096, rev_cap=64, seed=0, entry=0,
                        stream=None) -> None:
    """Incremental build (insertion waves) of the index's graph; entry 0 = entry points by
    id, 1 = by attributes; see include/nhq.h."""
    _check(load_library().nhq_index_build_nsw(index, degree, L, wave_max, rev_cap, entry,
                                              C.c_uint64(int(seed) & (2**64 - 1)),
                                              _stream(stream)))


def nhq_edge_select(index, cand_ids, R, nbr_out, stream=None) -> None:
    N = nhq_index_info(index)[0]
    L = _shape(cand_ids)[1]
    _check(load_library().nhq_edge_select(index, _ptr(cand_ids, np.uint32, (N, L), "cand_ids"),
                                          L, R, _ptr(nbr_out, np.uint32, (N, R), "nbr_out"),
                                          _stream(stream)))


def nhq_reverse_candidates(index, nbr, cap, out, stream=None) -> None:
    N = nhq_index_info(index)[0]
    R = _shape(nbr)[1]
    _check(load_library().nhq_reverse_candidates(index, _ptr(nbr, np.uint32, (N, R), "nbr"), R,
                                                 cap, _ptr(out, np.uint32, (N, R + cap), "out"),
                                                 _stream(stream)))


def nhq_index_set_graph(index, nbr, stream=None) -> None:
    N = nhq_index_info(index)[0]
    R = _shape(nbr)[1]
    _check(load_library().nhq_index_set_graph(index, _ptr(nbr, np.uint32, (N, R), "nbr"), R,
                                              _stream(stream)))


def nhq_index_get_graph(index, nbr, stream=None) -> None:
    N, _, _, R = nhq_index_info(index)
    _check(load_library().nhq_index_get_graph(index, _ptr(nbr, np.uint32, (N, R), "nbr"),
                                              _stream(stream)))


def _build_params(K, reverse, reverse_cap, knn_dtype=0):
    return _BuildParams(int(K), int(reverse), int(reverse_cap), int(knn_dtype))


def nhq_index_build(index, degree, K=64, reverse=1, reverse_cap=64, knn_dtype=0,
                    stream=None) -> None:
    p = _build_params(K, reverse, reverse_cap, knn_dtype)
    _check(load_library().nhq_index_build(index, degree, C.byref(p), _stream(stream)))


def nhq_build(vectors, attributes, degree, weights=None, K=64, reverse=1, reverse_cap=64,
              knn_dtype=0, stream=None) -> int:
    N, d = _shape(vectors)
    m = _shape(attributes)[1]
    p = _build_params(K, reverse, reverse_cap, knn_dtype)
    out = C.c_void_p()
    dt, vp = _vec_ptr(vectors, N, d)
    if dt == F32:
        _check(load_library().nhq_build(vp, N, d,
                                         _ptr(attributes, np.uint8, (N, m), "attributes"), m,
                                         degree, _weights(weights), C.byref(p), _stream(stream),
                                         C.byref(out)))
    else:
        _check(load_library().nhq_build_typed(vp, dt, N, d,
                                               _ptr(attributes, np.uint8, (N, m), "attributes"),
                                               m, degree, _weights(weights), C.byref(p),
                                               _stream(stream), C.byref(out)))
    return out.value


def nhq_build_typed(vectors, attributes, degree, weights=None, K=64, reverse=1, reverse_cap=64,
                    knn_dtype=0, stream=None) -> int:
    """nhq_build for f32, f16 or bf16 vectors (the type is taken from the array)."""
    return nhq_build(vectors, attributes, degree, weights, K, reverse, reverse_cap, knn_dtype,
                     stream)


def nhq_postfilter(ids, dists, chi, k_out, out_ids, out_dists, stream=None) -> None:
    """Keep the records with chi = 0 of each row of ids/dists/chi [Q, k_in], in order,
    into out_ids/out_dists [Q, k_out] (the post-filter strategy)."""
    Q, k_in = _shape(ids)
    _check(load_library().nhq_postfilter(
        Q, k_in, k_out, _ptr(ids, np.uint32, (Q, k_in), "ids"),
        _ptr(dists, np.float32, (Q, k_in), "dists"), _ptr(chi, np.uint8, (Q, k_in), "chi"),
        _ptr(out_ids, np.uint32, (Q, k_out), "out_ids"),
        _ptr(out_dists, np.float32, (Q, k_out), "out_dists"), _stream(stream)))


def nhq_merge_topk(ids, dists, offsets, k_out, out_ids, out_dists, chi=None, out_chi=None,
                   stream=None) -> None:
    """Merge per-shard top-k lists ids/dists [P, Q, k_in] (shard-local ids, global id =
    offsets[p] + local) into out_ids/out_dists [Q, k_out] by (Gamma, global id)."""
    P, Q, k_in = _shape(ids)
    _check(load_library().nhq_merge_topk(
        P, Q, k_in, k_out, _ptr(ids, np.uint32, (P, Q, k_in), "ids"),
        _ptr(dists, np.float32, (P, Q, k_in), "dists"), _ptr(chi, np.uint8, (P, Q, k_in), "chi"),
        _ptr(offsets, np.uint32, (P,), "offsets"), _ptr(out_ids, np.uint32, (Q, k_out), "out_ids"),
        _ptr(out_dists, np.float32, (Q, k_out), "out_dists"),
        _ptr(out_chi, np.uint8, (Q, k_out), "out_chi"), _stream(stream)))


def nhq_brute_force(index, queries, query_attributes, k, ids, dists=None, chi=None,
                    weights="index", stream=None, wildcard=0) -> None:
    """``wildcard=1``: a query code 255 leaves its attribute unconstrained."""
    Q, d = _shape(queries)
    m = _shape(query_attributes)[1]
    w = None if weights == "index" else C.byref(_weights(weights))
    _check(load_library().nhq_brute_force_wildcard(
        index, _ptr(queries, np.float32, (Q, d), "queries"),
        _ptr(query_attributes, np.uint8, (Q, m), "query_attributes"), Q, k, w, int(wildcard),
        _ptr(ids, np.uint32, (Q, k), "ids"), _ptr(dists, np.float32, (Q, k), "dists"),
        _ptr(chi, np.uint8, (Q, k), "chi"), _stream(stream)))


def nhq_brute_force_wildcard(index, queries, query_attributes, k, wildcard, ids, dists=None,
                             chi=None, weights="index", stream=None) -> None:
    nhq_brute_force(index, queries, query_attributes, k, ids, dists, chi, weights, stream,
                    wildcard)


def _search_params(seed, h, max_iters, warps_per_block, hash_bits, vec_dtype, rerank,
                   seed_mode=SEED_RANDOM, seeds=None, Q=None, stop_model=None,
                   stop_threshold=0.5, stop_min=0, stop_every=1, wildcard=0,
                   warps_per_query=0, entry_model=None, entry_cells=0, cells_out=None,
                   tile_rows=0):
    """Search parameters; ``seeds`` ([Q][n] uint32, 0xFFFFFFFF = none) selects SEED_GIVEN;
    ``stop_model`` (device f32 [MLP_PARAMS]) turns on the learned early stop."""
    n_seeds, sp = 0, None
    if seeds is not None:
        seed_mode = SEED_GIVEN
        n_seeds = _shape(seeds)[1]
        sp = _ptr(seeds, np.uint32, (Q, n_seeds), "seeds")
    mp = _ptr(stop_model, np.float32, (MLP_PARAMS,), "stop_model")
    ep = _ptr(entry_model, np.float32, None, "entry_model")
    cp = _ptr(cells_out, np.int32, None, "cells_out")
    return _SearchParams(int(seed) & (2**64 - 1), int(h), int(max_iters), int(warps_per_block),
                         int(hash_bits), int(vec_dtype), int(rerank), int(seed_mode),
                         int(n_seeds), sp, mp, float(stop_threshold), int(stop_min),
                         int(stop_every), int(wildcard), int(warps_per_query), ep,
                         int(entry_cells), cp, int(tile_rows))


def nhq_search(index, queries, query_attributes, k, ef, ids, dists=None, chi=None, status=None,
               ndc=None, expansions=None, h=1, seed=0, max_iters=0, warps_per_block=0,
               hash_bits=0, vec_dtype=VEC_F32, rerank=0, seed_mode=SEED_RANDOM, seeds=None,
               stop_model=None, stop_threshold=0.5, stop_min=0, stop_every=1,
               stream=None, wildcard=0, warps_per_query=0, entry_model=None, entry_cells=0,
               cells_out=None, tile_rows=0) -> None:
    Q, d = _shape(queries)
    m = _shape(query_attributes)[1]
    p = _search_params(seed, h, max_iters, warps_per_block, hash_bits, vec_dtype, rerank,
                       seed_mode, seeds, Q, stop_model, stop_threshold, stop_min, stop_every,
                       wildcard, warps_per_query, entry_model, entry_cells, cells_out,
                       tile_rows)
    _check(load_library().nhq_search(
        index, _ptr(queries, np.float32, (Q, d), "queries"),
        _ptr(query_attributes, np.uint8, (Q, m), "query_attributes"), Q, k, ef, C.byref(p),
        _ptr(ids, np.uint32, (Q, k), "ids"), _ptr(dists, np.float32, (Q, k), "dists"),
        _ptr(chi, np.uint8, (Q, k), "chi"), _ptr(status, np.int32, (Q,), "status"),
        _ptr(ndc, np.int32, (Q,), "ndc"), _ptr(expansions, np.int32, (Q,), "expansions"),
        _stream(stream)))


def nhq_search_batched(index, queries, query_attributes, k_arr, ef_arr, k_max, ids, dists=None,
                       chi=None, status=None, ndc=None, expansions=None, h=1, seed=0,
                       max_iters=0, warps_per_block=0, hash_bits=0, vec_dtype=VEC_F32, rerank=0,
                       seed_mode=SEED_RANDOM, seeds=None, stream=None, wildcard=0,
                       warps_per_query=0, entry_model=None, entry_cells=0,
                       tile_rows=0) -> None:
    Q, d = _shape(queries)
    m = _shape(query_attributes)[1]
    p = _search_params(seed, h, max_iters, warps_per_block, hash_bits, vec_dtype, rerank,
                       seed_mode, seeds, Q, wildcard=wildcard, warps_per_query=warps_per_query,
                       entry_model=entry_model, entry_cells=entry_cells, tile_rows=tile_rows)
    _check(load_library().nhq_search_batched(
        index, _ptr(queries, np.float32, (Q, d), "queries"),
        _ptr(query_attributes, np.uint8, (Q, m), "query_attributes"), Q,
        _ptr(k_arr, np.int32, (Q,), "k_arr"), _ptr(ef_arr, np.int32, (Q,), "ef_arr"), k_max,
        C.byref(p), _ptr(ids, np.uint32, (Q, k_max), "ids"),
        _ptr(dists, np.float32, (Q, k_max), "dists"), _ptr(chi, np.uint8, (Q, k_max), "chi"),
        _ptr(status, np.int32, (Q,), "status"), _ptr(ndc, np.int32, (Q,), "ndc"),
        _ptr(expansions, np.int32, (Q,), "expansions"), _stream(stream)))


def nhq_brute_force_noalloc(vectors, packed_attributes, m, queries, packed_query_attributes, k,
                            ids, dists=None, chi=None, weights=None, stream=None) -> None:
    """Allocation-free brute-force top-k for callers that cannot allocate device
    memory at call time; every array is a device tensor and ``m`` is the number of
    attributes packed into each u32 word (see include/nhq.h)."""
    N, d = _shape(vectors)
    Q = _shape(queries)[0]
    _check(load_library().nhq_brute_force_noalloc(
        _ptr(vectors, np.float32, (N, d), "vectors"),
        _ptr(packed_attributes, np.uint32, (N,), "packed_attributes"), N, d, int(m),
        _ptr(queries, np.float32, (Q, d), "queries"),
        _ptr(packed_query_attributes, np.uint32, (Q,), "packed_query_attributes"), Q, k,
        _weights(weights), _ptr(ids, np.uint32, (Q, k), "ids"),
        _ptr(dists, np.float32, (Q, k), "dists"), _ptr(chi, np.uint8, (Q, k), "chi"),
        _stream(stream)))


def nhq_autotune_search(index, queries, query_attributes, k, ef, ids, h=1, seed=0,
                        vec_dtype=VEC_F32, rerank=0, seed_mode=SEED_RANDOM, stream=None,
                        return_wpq=False):
    """Fastest result-preserving launch shape for this batch; returns
    (warps_per_block, hash_bits, ms_per_call), with warps_per_query first when
    ``return_wpq``."""
    Q, d = _shape(queries)
    m = _shape(query_attributes)[1]
    p = _search_params(seed, h, 0, 0, 0, vec_dtype, rerank, seed_mode, None, Q)
    ms = C.c_float(0.0)
    _check(load_library().nhq_autotune_search(
        index, _ptr(queries, np.float32, (Q, d), "queries"),
        _ptr(query_attributes, np.uint8, (Q, m), "query_attributes"), Q, k, ef, C.byref(p),
        _ptr(ids, np.uint32, (Q, k), "ids"), C.byref(ms), _stream(stream)))
    if return_wpq:
        return p.warps_per_query, p.warps_per_block, p.hash_bits, ms.value
    return p.warps_per_block, p.hash_bits, ms.value


def nhq_autotune(index, queries, query_attributes, k, ef, ids, stream=None, **kw):
    """nhq_autotune_search returning every tuned field: dict(warps_per_query, tile_rows,
    warps_per_block, hash_bits, ms); ``kw`` as nhq_search (seed, h, vec_dtype, rerank,
    seed_mode, entry_model, entry_cells, stop_model, ...)."""
    Q, d = _shape(queries)
    m = _shape(query_attributes)[1]
    p = _search_params(kw.get("seed", 0), kw.get("h", 1), kw.get("max_iters", 0), 0, 0,
                       kw.get("vec_dtype", VEC_F32), kw.get("rerank", 0),
                       kw.get("seed_mode", SEED_RANDOM), None, Q, kw.get("stop_model"),
                       kw.get("stop_threshold", 0.5), kw.get("stop_min", 0),
                       kw.get("stop_every", 1), kw.get("wildcard", 0), 0,
                       kw.get("entry_model"), kw.get("entry_cells", 0))
    ms = C.c_float(0.0)
    _check(load_library().nhq_autotune_search(
        index, _ptr(queries, np.float32, (Q, d), "queries"),
        _ptr(query_attributes, np.uint8, (Q, m), "query_attributes"), Q, k, ef, C.byref(p),
        _ptr(ids, np.uint32, (Q, k), "ids"), C.byref(ms), _stream(stream)))
    return dict(warps_per_query=p.warps_per_query, tile_rows=p.tile_rows,
                warps_per_block=p.warps_per_block, hash_bits=p.hash_bits, ms=ms.value)


def nhq_index_build_cells(index, E, stream=None) -> None:
    _check(load_library().nhq_index_build_cells(index, int(E), _stream(stream)))


def nhq_index_cells(index, cell_of=None, stream=None) -> int:
    """Number of entry cells; fills cell_of [N] (uint32) when given."""
    E = C.c_int32(0)
    n = _shape(cell_of)[0] if cell_of is not None else None
    _check(load_library().nhq_index_cells(index, C.byref(E),
                                          _ptr(cell_of, np.uint32, (n,) if n else None,
                                               "cell_of"), _stream(stream)))
    return E.value


def nhq_entry_param_count(d, E) -> int:
    return int(load_library().nhq_entry_param_count(int(d), int(E)))


def nhq_entry_forward(params, E, queries, logits, stream=None) -> None:
    n, d = _shape(queries)
    _check(load_library().nhq_entry_forward(
        _ptr(params, np.float32, (nhq_entry_param_count(d, E),), "params"), d, int(E),
        _ptr(queries, np.float32, (n, d), "queries"), n,
        _ptr(logits, np.float32, (n, E), "logits"), _stream(stream)))


def nhq_entry_grad(params, E, queries, labels, grad, loss, stream=None) -> None:
    n, d = _shape(queries)
    np_ = nhq_entry_param_count(d, E)
    _check(load_library().nhq_entry_grad(
        _ptr(params, np.float32, (np_,), "params"), d, int(E),
        _ptr(queries, np.float32, (n, d), "queries"), _ptr(labels, np.int32, (n,), "labels"), n,
        _ptr(grad, np.float32, (np_,), "grad"), _ptr(loss, np.float32, (1,), "loss"),
        _stream(stream)))


def nhq_entry_train(params, E, queries, labels, epochs=4, batch=1024, lr=1e-3,
                    stream=None) -> None:
    n, d = _shape(queries)
    _check(load_library().nhq_entry_train(
        _ptr(params, np.float32, (nhq_entry_param_count(d, E),), "params"), d, int(E),
        _ptr(queries, np.float32, (n, d), "queries"), _ptr(labels, np.int32, (n,), "labels"), n,
        int(epochs), int(batch), float(lr), _stream(stream)))


def nhq_entry_labels(index, ids, labels, stream=None) -> None:
    n, k = _shape(ids)
    _check(load_library().nhq_entry_labels(index, _ptr(ids, np.uint32, (n, k), "ids"), k, n,
                                           _ptr(labels, np.int32, (n,), "labels"),
                                           _stream(stream)))


def nhq_autotune_batched(index, queries, query_attributes, k_arr, ef_arr, k_max, ids,
                         stream=None, **kw):
    """nhq_autotune_search for a heterogeneous batch (device k_arr / ef_arr); returns
    dict(warps_per_query, tile_rows, warps_per_block, hash_bits, ms)."""
    Q, d = _shape(queries)
    m = _shape(query_attributes)[1]
    p = _search_params(kw.get("seed", 0), kw.get("h", 1), kw.get("max_iters", 0), 0, 0,
                       kw.get("vec_dtype", VEC_F32), kw.get("rerank", 0),
                       kw.get("seed_mode", SEED_RANDOM), None, Q,
                       wildcard=kw.get("wildcard", 0))
    ms = C.c_float(0.0)
    _check(load_library().nhq_autotune_batched(
        index, _ptr(queries, np.float32, (Q, d), "queries"),
        _ptr(query_attributes, np.uint8, (Q, m), "query_attributes"), Q,
        _ptr(k_arr, np.int32, (Q,), "k_arr"), _ptr(ef_arr, np.int32, (Q,), "ef_arr"), k_max,
        C.byref(p), _ptr(ids, np.uint32, (Q, k_max), "ids"), C.byref(ms), _stream(stream)))
    return dict(warps_per_query=p.warps_per_query, tile_rows=p.tile_rows,
                warps_per_block=p.warps_per_block, hash_bits=p.hash_bits, ms=ms.value)


def nhq_recall(ids, truth, stream=None) -> float:
    """Mean recall (Eq. 3) of ids [Q, k] against truth [Q, k_truth] (device uint32,
    0xFFFFFFFF entries of truth not counted; queries without truth skipped)."""
    Q, k = _shape(ids)
    kt = _shape(truth)[1]
    r = C.c_float(0.0)
    _check(load_library().nhq_recall(_ptr(ids, np.uint32, (Q, k), "ids"), k,
                                     _ptr(truth, np.uint32, (Q, kt), "truth"), kt, Q,
                                     C.byref(r), _stream(stream)))
    return r.value


def nhq_autotune_beam(index, queries, query_attributes, k, ef_list, truth, target, ids, h=1,
                      seed=0, vec_dtype=VEC_F32, rerank=0, seed_mode=SEED_RANDOM, stream=None):
    """Smallest ef of ef_list reaching ``target`` recall against truth [Q, k], then the
    fastest launch shape for it; returns dict(ef, recall, warps_per_query,
    warps_per_block, hash_bits, ms)."""
    Q, d = _shape(queries)
    m = _shape(query_attributes)[1]
    efs = (C.c_int32 * len(ef_list))(*[int(e) for e in ef_list])
    p = _search_params(seed, h, 0, 0, 0, vec_dtype, rerank, seed_mode, None, Q)
    ef, rec, ms = C.c_int32(0), C.c_float(0.0), C.c_float(0.0)
    _check(load_library().nhq_autotune_beam(
        index, _ptr(queries, np.float32, (Q, d), "queries"),
        _ptr(query_attributes, np.uint8, (Q, m), "query_attributes"), Q, k,
        C.cast(efs, C.c_void_p), len(ef_list), _ptr(truth, np.uint32, (Q, k), "truth"),
        float(target), C.byref(p), _ptr(ids, np.uint32, (Q, k), "ids"), C.byref(ef),
        C.byref(rec), C.byref(ms), _stream(stream)))
    return dict(ef=ef.value, recall=rec.value, warps_per_query=p.warps_per_query,
                tile_rows=p.tile_rows, warps_per_block=p.warps_per_block,
                hash_bits=p.hash_bits, ms=ms.value)


class SearchGraph:
    """A captured nhq_search call (see nhq_search_graph_create); replays with launch()."""

    def __init__(self, index, queries, query_attributes, k, ef, ids, dists=None, chi=None, **kw):
        Q, d = _shape(queries)
        m = _shape(query_attributes)[1]
        kw.setdefault("seed_mode", SEED_RANDOM)
        self._p = _search_params(kw.get("seed", 0), kw.get("h", 1), kw.get("max_iters", 0),
                                 kw.get("warps_per_block", 0), kw.get("hash_bits", 0),
                                 kw.get("vec_dtype", VEC_F32), kw.get("rerank", 0),
                                 kw["seed_mode"], None, Q, wildcard=kw.get("wildcard", 0),
                                 warps_per_query=kw.get("warps_per_query", 0),
                                 tile_rows=kw.get("tile_rows", 0))
        out = C.c_void_p()
        _check(load_library().nhq_search_graph_create(
            index, _ptr(queries, np.float32, (Q, d), "queries"),
            _ptr(query_attributes, np.uint8, (Q, m), "query_attributes"), Q, k, ef,
            C.byref(self._p), _ptr(ids, np.uint32, (Q, k), "ids"),
            _ptr(dists, np.float32, (Q, k), "dists"), _ptr(chi, np.uint8, (Q, k), "chi"),
            C.byref(out)))
        self.handle = out.value

    def launch(self, stream=None):
        _check(load_library().nhq_search_graph_launch(self.handle, _stream(stream)))

    def close(self):
        if self.handle:
            load_library().nhq_search_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nhq_search_graph_create(*a, **kw):
    return SearchGraph(*a, **kw)


class BatchedSearchGraph(SearchGraph):
    """A captured nhq_search_batched call (nhq_search_graph_create_batched)."""

    def __init__(self, index, queries, query_attributes, k_arr, ef_arr, k_max, ids,
                 dists=None, chi=None, **kw):
        Q, d = _shape(queries)
        m = _shape(query_attributes)[1]
        self._p = _search_params(kw.get("seed", 0), kw.get("h", 1), kw.get("max_iters", 0),
                                 kw.get("warps_per_block", 0), kw.get("hash_bits", 0),
                                 kw.get("vec_dtype", VEC_F32), kw.get("rerank", 0),
                                 kw.get("seed_mode", SEED_RANDOM), None, Q,
                                 wildcard=kw.get("wildcard", 0),
                                 warps_per_query=kw.get("warps_per_query", 0),
                                 tile_rows=kw.get("tile_rows", 0))
        out = C.c_void_p()
        _check(load_library().nhq_search_graph_create_batched(
            index, _ptr(queries, np.float32, (Q, d), "queries"),
            _ptr(query_attributes, np.uint8, (Q, m), "query_attributes"), Q,
            _ptr(k_arr, np.int32, (Q,), "k_arr"), _ptr(ef_arr, np.int32, (Q,), "ef_arr"),
            k_max, C.byref(self._p), _ptr(ids, np.uint32, (Q, k_max), "ids"),
            _ptr(dists, np.float32, (Q, k_max), "dists"), _ptr(chi, np.uint8, (Q, k_max), "chi"),
            C.byref(out)))
        self.handle = out.value


def nhq_search_graph_create_batched(*a, **kw):
    return BatchedSearchGraph(*a, **kw)


def nhq_search_graph_launch(graph, stream=None):
    graph.launch(stream)


def nhq_search_graph_free(graph):
    graph.close()


def nhq_search_trace(index, queries, query_attributes, k, ef, features, labels, query,
                     stop_min=0, stop_every=1, h=1, seed=0, seed_mode=SEED_RANDOM,
                     vec_dtype=VEC_F32, stream=None) -> int:
    """Training records for the learned stop (device arrays); returns their count."""
    Q, d = _shape(queries)
    m = _shape(query_attributes)[1]
    cap = _shape(labels)[0]
    p = _search_params(seed, h, 0, 0, 0, vec_dtype, 0, seed_mode, None, Q, None, 0.5, stop_min,
                       stop_every)
    n = C.c_int64(0)
    _check(load_library().nhq_search_trace(
        index, _ptr(queries, np.float32, (Q, d), "queries"),
        _ptr(query_attributes, np.uint8, (Q, m), "query_attributes"), Q, k, ef, C.byref(p),
        _ptr(features, np.float32, (cap, MLP_INPUTS), "features"),
        _ptr(labels, np.uint8, (cap,), "labels"), _ptr(query, np.int32, (cap,), "query"), cap,
        C.byref(n), _stream(stream)))
    return n.value


def nhq_mlp_forward(params, features, logits, stream=None) -> None:
    n = _shape(features)[0]
    _check(load_library().nhq_mlp_forward(_ptr(params, np.float32, (MLP_PARAMS,), "params"),
                                          _ptr(features, np.float32, (n, MLP_INPUTS), "features"),
                                          n, _ptr(logits, np.float32, (n,), "logits"),
                                          _stream(stream)))


def nhq_mlp_grad(params, features, labels, grad, loss, stream=None) -> None:
    n = _shape(features)[0]
    _check(load_library().nhq_mlp_grad(_ptr(params, np.float32, (MLP_PARAMS,), "params"),
                                       _ptr(features, np.float32, (n, MLP_INPUTS), "features"),
                                       _ptr(labels, np.float32, (n,), "labels"), n,
                                       _ptr(grad, np.float32, (MLP_PARAMS,), "grad"),
                                       _ptr(loss, np.float32, (1,), "loss"), _stream(stream)))


def nhq_mlp_train(params, features, labels, epochs=3, batch=4096, lr=1e-3, stream=None) -> None:
    n = _shape(features)[0]
    _check(load_library().nhq_mlp_train(_ptr(params, np.float32, (MLP_PARAMS,), "params"),
                                        _ptr(features, np.float32, (n, MLP_INPUTS), "features"),
                                        _ptr(labels, np.float32, (n,), "labels"), n, epochs,
                                        batch, float(lr), _stream(stream)))


def nhq_save(index, path) -> None:
    _check(load_library().nhq_save(index, os.fsencode(path)))


def nhq_load(path, stream=None) -> int:
    out = C.c_void_p()
    _check(load_library().nhq_load(os.fsencode(path), _stream(stream), C.byref(out)))
    return out.value


class Index:
    """Owning wrapper around an nhq_index handle (freed on close / context exit)."""

    def __init__(self, handle):
        self.handle = handle

    @classmethod
    def create(cls, vectors, attributes, weights=None, stream=None):
        if _vec_dtype_of(vectors)[0] != F32:
            return cls(nhq_index_create_typed(vectors, attributes, weights, stream))
        return cls(nhq_index_create(vectors, attributes, weights, stream))

    @classmethod
    def build(cls, vectors, attributes, degree=32, weights=None, K=64, reverse=1,
              reverse_cap=64, knn_dtype=0, stream=None):
        return cls(nhq_build(vectors, attributes, degree, weights, K, reverse, reverse_cap,
                             knn_dtype, stream))

    @property
    def info(self):
        return nhq_index_info(self.handle)

    def close(self):
        if self.handle:
            nhq_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
