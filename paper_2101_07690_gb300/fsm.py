"""Python binding of the C ABI in include/fsm.h (argument marshalling only).

Every function keeps the C name and forwards to ``_build/libfsm.so``; all mining work runs in
the library's CUDA kernels.  A missing library raises ``ImportError`` -- there is no other
implementation to fall back to.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfsm.so")

FSM_OK = 0
FSM_EINVAL = -1
FSM_ENOMEM = -2
FSM_ECUDA = -3
FSM_ETIMEOUT = -4
FSM_EUNSUPPORTED = -5
_NAMES = {FSM_EINVAL: "FSM_EINVAL", FSM_ENOMEM: "FSM_ENOMEM", FSM_ECUDA: "FSM_ECUDA",
          FSM_ETIMEOUT: "FSM_ETIMEOUT", FSM_EUNSUPPORTED: "FSM_EUNSUPPORTED"}

# every entry point that include/fsm.h declares
EXPORTS = ["fsm_load_graph", "fsm_set_option", "fsm_mine", "fsm_result_count", "fsm_result_get",
           "fsm_result_embeddings", "fsm_result_copy", "fsm_result_pairs", "fsm_result_stat", "fsm_free_result",
           "fsm_free_graph", "fsm_last_error", "fsm_debug_dissect", "fsm_edge_supports_noalloc",
           "fsm_result_exact", "fsm_result_features", "fsm_mlp_create", "fsm_mlp_set_params",
           "fsm_mlp_get_params", "fsm_mlp_set_norm", "fsm_mlp_fit_norm", "fsm_mlp_gradients", "fsm_mlp_train",
           "fsm_mlp_predict", "fsm_mlp_predict_device", "fsm_mlp_free"]

MLP_NPARAM = 32 * 64 + 64 + 64 * 64 + 64 + 64 + 1


class FsmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str | None = None):
    """Load libfsm.so (built by ``paper_2101_07690_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libfsm.so not built at {p}; run paper_2101_07690_gb300.build.build()")
    lib = ctypes.CDLL(p)
    P = ctypes.POINTER
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "fsm_load_graph": (ctypes.c_int, [P(i32), P(i32), P(i32), i32, i32, P(vp)]),
        "fsm_set_option": (ctypes.c_int, [vp, ctypes.c_char_p, i64]),
        "fsm_mine": (ctypes.c_int, [vp, i32, i64, ctypes.c_double, P(vp)]),
        "fsm_result_count": (i64, [vp]),
        "fsm_result_get": (ctypes.c_int, [vp, i64, P(i32), P(u64), P(i64)]),
        "fsm_result_embeddings": (ctypes.c_int, [vp, i64, P(i64)]),
        "fsm_result_copy": (ctypes.c_int, [vp, P(i32), P(u64), P(i64), P(i64)]),
        "fsm_result_pairs": (ctypes.c_int, [vp, P(u64)]),
        "fsm_result_stat": (ctypes.c_int, [vp, ctypes.c_char_p, P(i64)]),
        "fsm_free_result": (None, [vp]),
        "fsm_free_graph": (None, [vp]),
        "fsm_last_error": (ctypes.c_char_p, []),
        "fsm_debug_dissect": (ctypes.c_int, [i32, P(i32), P(ctypes.c_uint32), P(ctypes.c_uint32), P(i32), P(i32)]),
        "fsm_edge_supports_noalloc": (ctypes.c_int, [vp, vp, vp, i32, i32, vp, vp, vp]),
        "fsm_result_exact": (ctypes.c_int, [vp, P(i32)]),
        "fsm_result_features": (ctypes.c_int, [vp, P(ctypes.c_float)]),
        "fsm_mlp_create": (ctypes.c_int, [u64, P(vp)]),
        "fsm_mlp_set_params": (ctypes.c_int, [vp, P(ctypes.c_float)]),
        "fsm_mlp_get_params": (ctypes.c_int, [vp, P(ctypes.c_float)]),
        "fsm_mlp_set_norm": (ctypes.c_int, [vp, P(ctypes.c_float), P(ctypes.c_float)]),
        "fsm_mlp_fit_norm": (ctypes.c_int, [vp, P(ctypes.c_float), i64]),
        "fsm_mlp_gradients": (ctypes.c_int, [vp, P(ctypes.c_float), P(ctypes.c_float), i64, P(ctypes.c_float),
                                             P(ctypes.c_float)]),
        "fsm_mlp_train": (ctypes.c_int, [vp, P(ctypes.c_float), P(ctypes.c_float), i64, i32, i32, ctypes.c_float,
                                         u64, P(ctypes.c_float)]),
        "fsm_mlp_predict": (ctypes.c_int, [vp, P(ctypes.c_float), i64, P(ctypes.c_float)]),
        "fsm_mlp_predict_device": (ctypes.c_int, [vp, vp, i64, vp, vp]),
        "fsm_mlp_free": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != FSM_OK:
        raise FsmError(rc, fsm_last_error())
    return rc


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def fsm_last_error() -> str:
    return (load().fsm_last_error() or b"").decode()


def fsm_load_graph(row_ptr, col, labels, n: int, num_labels: int) -> int:
    """Copy a CSR graph to the current device; returns the graph handle.  Arrays may be numpy
    arrays or raw host addresses (ints) of int32 buffers."""
    lib = load()
    keep = []

    def arg(a):
        if isinstance(a, int):
            return ctypes.cast(a, ctypes.POINTER(ctypes.c_int32))
        arr = _i32(a)
        keep.append(arr)
        return _ptr(arr, ctypes.c_int32)

    h = ctypes.c_void_p()
    _check(lib.fsm_load_graph(arg(row_ptr), arg(col), arg(labels), int(n), int(num_labels), ctypes.byref(h)))
    return h.value


def fsm_set_option(g: int, key: str, value: int) -> None:
    _check(load().fsm_set_option(g, key.encode(), int(value)))


def fsm_mine(g: int, k: int, min_support: int, sample_rate: float = 1.0) -> int:
    r = ctypes.c_void_p()
    _check(load().fsm_mine(g, int(k), int(min_support), float(sample_rate), ctypes.byref(r)))
    return r.value


def fsm_result_count(r: int) -> int:
    n = load().fsm_result_count(r)
    if n < 0:
        raise FsmError(int(n), fsm_last_error())
    return int(n)


def fsm_result_get(r: int, i: int, k: int):
    labels = np.zeros(k, np.int32)
    adj = ctypes.c_uint64()
    sup = ctypes.c_int64()
    _check(load().fsm_result_get(r, int(i), _ptr(labels, ctypes.c_int32), ctypes.byref(adj), ctypes.byref(sup)))
    return labels, int(adj.value), int(sup.value)


def fsm_result_embeddings(r: int, i: int) -> int:
    c = ctypes.c_int64()
    _check(load().fsm_result_embeddings(r, int(i), ctypes.byref(c)))
    return int(c.value)


def fsm_result_pairs(r: int) -> np.ndarray:
    """Pair bits of every pattern: bit q set when pair q of (0,1), (0,2), ... is an edge."""
    out = np.zeros(fsm_result_count(r), np.uint64)
    _check(load().fsm_result_pairs(r, _ptr(out, ctypes.c_uint64)))
    return out


def adj_from_pairs(pairs, k: int) -> np.ndarray:
    """Bit (i*k + j) words from pair bits: uint64 for k <= 8, Python ints (object array) for
    k = 9, whose bits run past 64."""
    pos = [i * k + j for i in range(k) for j in range(i + 1, k)]
    out = [sum(1 << pos[q] for q in range(len(pos)) if (int(w) >> q) & 1) for w in pairs]
    return np.array(out, dtype=np.uint64 if k <= 8 else object)


def fsm_result_copy(r: int, k: int) -> dict:
    """labels (n, k), adj (bit i*k + j; Python ints for k = 9), support, count."""
    n = fsm_result_count(r)
    out = {"labels": np.zeros((n, k), np.int32), "adj": np.zeros(n, np.uint64),
           "support": np.zeros(n, np.int64), "count": np.zeros(n, np.int64)}
    wide = k > 8
    _check(load().fsm_result_copy(r, _ptr(out["labels"], ctypes.c_int32),
                                  None if wide else _ptr(out["adj"], ctypes.c_uint64),
                                  _ptr(out["support"], ctypes.c_int64), _ptr(out["count"], ctypes.c_int64)))
    if wide:
        out["adj"] = adj_from_pairs(fsm_result_pairs(r), k)
    return out


def fsm_result_stat(r: int, key: str) -> int:
    v = ctypes.c_int64()
    _check(load().fsm_result_stat(r, key.encode(), ctypes.byref(v)))
    return int(v.value)


def fsm_free_result(r: int) -> None:
    if r:
        load().fsm_free_result(r)


def fsm_free_graph(g: int) -> None:
    if g:
        load().fsm_free_graph(g)


def fsm_debug_dissect(ids, adj_rows):
    """Host build of the dissection rule: returns (l_mask, join, used_fallback)."""
    ids = _i32(ids)
    rows = np.ascontiguousarray(adj_rows, dtype=np.uint32)
    lm, jn, fb = ctypes.c_uint32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().fsm_debug_dissect(len(ids), _ptr(ids, ctypes.c_int32), _ptr(rows, ctypes.c_uint32),
                                    ctypes.byref(lm), ctypes.byref(jn), ctypes.byref(fb)))
    return int(lm.value), int(jn.value), int(fb.value)


def fsm_edge_supports_noalloc(d_row_ptr: int, d_col: int, d_labels: int, n: int, num_labels: int,
                              d_support: int, d_count: int, stream: int = 0) -> None:
    """Size-2 pattern supports without device allocation; every pointer is a device address
    (int), outputs uint64[num_labels * num_labels]."""
    _check(load().fsm_edge_supports_noalloc(d_row_ptr, d_col, d_labels, int(n), int(num_labels),
                                            d_support, d_count, stream or None))


def fsm_result_exact(r: int) -> np.ndarray:
    out = np.zeros(fsm_result_count(r), np.int32)
    _check(load().fsm_result_exact(r, _ptr(out, ctypes.c_int32)))
    return out


def fsm_result_features(r: int) -> np.ndarray:
    out = np.zeros((fsm_result_count(r), 32), np.float32)
    _check(load().fsm_result_features(r, _ptr(out, ctypes.c_float)))
    return out


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def fsm_mlp_create(seed: int = 0) -> int:
    m = ctypes.c_void_p()
    _check(load().fsm_mlp_create(int(seed), ctypes.byref(m)))
    return m.value


def fsm_mlp_set_params(m: int, params) -> None:
    p = _f32(params).reshape(MLP_NPARAM)
    _check(load().fsm_mlp_set_params(m, _ptr(p, ctypes.c_float)))


def fsm_mlp_get_params(m: int) -> np.ndarray:
    out = np.zeros(MLP_NPARAM, np.float32)
    _check(load().fsm_mlp_get_params(m, _ptr(out, ctypes.c_float)))
    return out


def fsm_mlp_set_norm(m: int, mean, stdev) -> None:
    mu, sd = _f32(mean).reshape(32), _f32(stdev).reshape(32)
    _check(load().fsm_mlp_set_norm(m, _ptr(mu, ctypes.c_float), _ptr(sd, ctypes.c_float)))


def fsm_mlp_fit_norm(m: int, X) -> None:
    X = _f32(X).reshape(-1, 32)
    _check(load().fsm_mlp_fit_norm(m, _ptr(X, ctypes.c_float), len(X)))


def fsm_mlp_gradients(m: int, X, Y):
    X, Y = _f32(X).reshape(-1, 32), _f32(Y).reshape(-1)
    g = np.zeros(MLP_NPARAM, np.float32)
    loss = ctypes.c_float()
    _check(load().fsm_mlp_gradients(m, _ptr(X, ctypes.c_float), _ptr(Y, ctypes.c_float), len(Y),
                                    _ptr(g, ctypes.c_float), ctypes.byref(loss)))
    return g, float(loss.value)


def fsm_mlp_train(m: int, X, Y, epochs: int, batch: int, lr: float, seed: int = 0) -> float:
    X, Y = _f32(X).reshape(-1, 32), _f32(Y).reshape(-1)
    loss = ctypes.c_float()
    _check(load().fsm_mlp_train(m, _ptr(X, ctypes.c_float), _ptr(Y, ctypes.c_float), len(Y), int(epochs),
                                int(batch), float(lr), int(seed), ctypes.byref(loss)))
    return float(loss.value)


def fsm_mlp_predict(m: int, X) -> np.ndarray:
    X = _f32(X).reshape(-1, 32)
    out = np.zeros(len(X), np.float32)
    _check(load().fsm_mlp_predict(m, _ptr(X, ctypes.c_float), len(X), _ptr(out, ctypes.c_float)))
    return out


def fsm_mlp_predict_device(m: int, d_X: int, n: int, d_out: int, stream: int = 0) -> None:
    _check(load().fsm_mlp_predict_device(m, d_X, int(n), d_out, stream or None))


def fsm_mlp_free(m: int) -> None:
    if m:
        load().fsm_mlp_free(m)


STATS = ["k", "levels", "pieces", "candidates", "embeddings", "final_embeddings", "quick_patterns", "patterns",
         "live_patterns", "frontier_max", "kernel_launches", "time_ns", "final_level_ns",
         "count_ns", "domain_ns", "emit_ns", "count_launches", "domain_launches", "emit_launches",
         "count_bytes", "domain_bytes", "emit_bytes", "fused_ns", "fused_launches", "fused_bytes",
         "sampled_candidates", "recount_patterns", "recount_frontier", "sampled_edges", "qp_grows", "fused_fallbacks", "fused_pool_words"] + [
             f"{p}_{f}_l{l}" for p in ("count", "domain", "emit", "fused") for f in ("ns", "launches", "bytes")
             for l in range(1, 7)] + [f"chunk_l{l}" for l in range(1, 7)] + [f"pieces_l{l}" for l in range(1, 7)]


class Graph:
    """Owning wrapper of a graph handle."""

    def __init__(self, row_ptr, col, labels, num_labels: int, mode: str = "edge"):
        self.n = int(len(labels))
        self.handle = fsm_load_graph(row_ptr, col, labels, self.n, int(num_labels))
        self.set_mode(mode)

    @classmethod
    def from_graphgen(cls, g, mode: str = "edge"):
        return cls(g.row_ptr, g.col, g.labels, g.num_labels, mode)

    def set_mode(self, mode: str):
        fsm_set_option(self.handle, "mode", {"edge": 0, "vertex": 1}[mode])

    def set_option(self, key: str, value: int):
        fsm_set_option(self.handle, key, value)

    def mine(self, k: int, t: int, sample_rate: float = 1.0, stats: bool = False, features: bool = False):
        r = fsm_mine(self.handle, k, t, sample_rate)
        try:
            out = fsm_result_copy(r, k)
            out["exact"] = fsm_result_exact(r)
            if features:
                out["features"] = fsm_result_features(r)
            if stats:
                out["stats"] = {s: fsm_result_stat(r, s) for s in STATS}
        finally:
            fsm_free_result(r)
        return out

    def close(self):
        if self.handle:
            fsm_free_graph(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
