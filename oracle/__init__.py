"""CPU oracle for exact frequent subgraph mining under MNI support.

TEST INFRASTRUCTURE ONLY: only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference legs may import this package.  The CUDA library never imports it and
shares no code with it.

``fsm_oracle.c`` is plain C (ESU enumeration of connected vertex sets, every connected edge
subset in edge-induced mode, brute-force canonical code over all k! permutations, MNI image
sets over every optimal permutation).  ``brute.py`` is a second, independent oracle for tiny
graphs that follows the MNI definition literally by enumerating injective maps.

Pattern encoding shared by both oracles' outputs (and by the library's C ABI, which defines
the same encoding independently):
  * ``labels[k]``: vertex labels in canonical order;
  * ``adj``: bit ``i*k + j`` (LSB = bit 0) set for each canonical edge i < j (a uint64 array for
    k <= 8; for k = 9, whose bits run past 64, an object array of Python ints);
  * patterns sorted ascending by the label sequence, then by the adjacency sequence
    A(0,1), A(0,2), ..., A(k-2,k-1) compared lexicographically (0 < 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "fsm_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no architecture flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            lib.oracle_mine.restype = ctypes.c_void_p
            lib.oracle_mine.argtypes = [ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32),
                                        P(ctypes.c_int32), ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64]
            lib.oracle_mine_sampled.restype = ctypes.c_void_p
            lib.oracle_mine_sampled.argtypes = lib.oracle_mine.argtypes + [ctypes.c_int32, ctypes.c_uint64,
                                                                           ctypes.c_double]
            lib.oracle_result_copy_sampled.restype = None
            lib.oracle_result_copy_sampled.argtypes = [ctypes.c_void_p, P(ctypes.c_int64), P(ctypes.c_int64)]
            lib.oracle_result_copy_sampled_domains.restype = None
            lib.oracle_result_copy_sampled_domains.argtypes = [ctypes.c_void_p, P(ctypes.c_int64),
                                                               P(ctypes.c_double)]
            lib.oracle_dissect.restype = ctypes.c_uint32
            lib.oracle_dissect.argtypes = [ctypes.c_int32, P(ctypes.c_uint32)]
            lib.oracle_mine_quota.restype = ctypes.c_void_p
            lib.oracle_mine_quota.argtypes = [ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32),
                                              P(ctypes.c_int32), ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                              ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64]
            lib.oracle_quota_draw.restype = None
            lib.oracle_quota_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, P(ctypes.c_uint64),
                                              P(ctypes.c_uint64)]
            lib.oracle_dissect_join.restype = ctypes.c_uint32
            lib.oracle_dissect_join.argtypes = [ctypes.c_int32, P(ctypes.c_uint32), P(ctypes.c_int32)]
            lib.oracle_edge_kept.restype = ctypes.c_int
            lib.oracle_edge_kept.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_int32, ctypes.c_int32]
            lib.oracle_kept.restype = ctypes.c_int
            lib.oracle_kept.argtypes = [ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_uint32), ctypes.c_uint64,
                                        ctypes.c_double]
            lib.oracle_result_count.restype = ctypes.c_int64
            lib.oracle_result_count.argtypes = [ctypes.c_void_p]
            lib.oracle_result_copy.restype = None
            lib.oracle_result_copy.argtypes = [ctypes.c_void_p, P(ctypes.c_int32), P(ctypes.c_uint64),
                                               P(ctypes.c_int64), P(ctypes.c_int64)]
            lib.oracle_free.restype = None
            lib.oracle_free.argtypes = [ctypes.c_void_p]
            lib.oracle_result_copy_pairs.restype = None
            lib.oracle_result_copy_pairs.argtypes = [ctypes.c_void_p, P(ctypes.c_uint64)]
            lib.oracle_pattern_support_rows.restype = ctypes.c_int
            lib.oracle_pattern_support_rows.argtypes = [ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32),
                                                        P(ctypes.c_int32), ctypes.c_int32, P(ctypes.c_int32),
                                                        P(ctypes.c_uint32), ctypes.c_int32, ctypes.c_int64,
                                                        P(ctypes.c_int64), P(ctypes.c_int64)]
            lib.oracle_pattern_support.restype = ctypes.c_int
            lib.oracle_pattern_support.argtypes = [ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_int32),
                                                   P(ctypes.c_int32), ctypes.c_int32, P(ctypes.c_int32),
                                                   ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64,
                                                   P(ctypes.c_int64), P(ctypes.c_int64)]
            _lib = lib
    return _lib


MODES = {"edge": 0, "vertex": 1}


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def adj_from_pairs(pairs, k: int):
    """``adj`` words (bit i*k + j) from pair words (bit q = pair q of (0,1), (0,2), ...,
    (k-2,k-1)): uint64 for k <= 8, Python ints (object array) for k = 9."""
    pos = [i * k + j for i in range(k) for j in range(i + 1, k)]
    out = [sum(1 << pos[q] for q in range(len(pos)) if (int(w) >> q) & 1) for w in pairs]
    return np.array(out, dtype=np.uint64 if k <= 8 else object)


def _result(lib, res, k: int) -> dict:
    npat = lib.oracle_result_count(res)
    out = {"labels": np.zeros((npat, k), np.int32), "adj": np.zeros(npat, np.uint64),
           "support": np.zeros(npat, np.int64), "count": np.zeros(npat, np.int64)}
    if npat:
        lib.oracle_result_copy(res, _ptr(out["labels"], ctypes.c_int32), _ptr(out["adj"], ctypes.c_uint64),
                               _ptr(out["support"], ctypes.c_int64), _ptr(out["count"], ctypes.c_int64))
    if k > 8:
        pairs = np.zeros(npat, np.uint64)
        if npat:
            lib.oracle_result_copy_pairs(res, _ptr(pairs, ctypes.c_uint64))
        out["adj"] = adj_from_pairs(pairs, k)
    return out


def mine(g, k: int, t: int, mode: str = "edge", roots: tuple[int, int] | None = None,
         max_embeddings: int = 0, sample: tuple[float, int] | None = None) -> dict:
    """All k-vertex patterns of graph ``g`` with MNI support >= t.

    ``roots=(b, e)`` restricts the enumeration to connected sets whose smallest vertex id is
    in [b, e); ``max_embeddings > 0`` stops after that many embeddings (roots taken in
    ascending order).  Both give a bounded sample of the work, whose supports are those of the
    sample.  ``sample=(p, seed)`` adds the statistics of sampled mining at rate p: directed
    edges are kept by a splitmix64 rule at rate sqrt(p), and an embedding is kept when the
    3-vertex part of its smallest-vertex-first dissection is made of kept edges as seen from
    the join vertex; ``ssupport`` and ``scount`` are the MNI support and embedding count over
    kept embeddings, ``spop[P, c]`` the size of canonical position c's sampled image set and
    ``sdeg[P, c]`` the sum of log(1 + degree) over it.
    Returns a dict of numpy arrays: labels (P, k) int32, adj (P,) (uint64, or Python ints for
    k = 9), support (P,) int64, count (P,) int64 (number of embeddings of each pattern)."""
    lib = _load()
    row_ptr = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    labels = np.ascontiguousarray(g.labels, dtype=np.int32)
    if labels.size and (labels.min() < 0 or labels.max() > 255):
        raise ValueError("oracle labels must lie in [0, 255]")
    b, e = (0, g.n) if roots is None else roots
    sp, sseed = (1.0, 0) if sample is None else sample
    res = lib.oracle_mine_sampled(g.n, _ptr(row_ptr, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                                  _ptr(labels, ctypes.c_int32), k, MODES[mode], int(t), int(b), int(e),
                                  int(max_embeddings), 1 if sample is not None else 0, int(sseed), float(sp))
    if not res:
        raise ValueError("oracle_mine rejected its arguments")
    try:
        out = _result(lib, res, k)
        npat = len(out["support"])
        if sample is not None:
            out["ssupport"] = np.zeros(npat, np.int64)
            out["scount"] = np.zeros(npat, np.int64)
            out["spop"] = np.zeros((npat, k), np.int64)
            out["sdeg"] = np.zeros((npat, k), np.float64)
            if npat:
                lib.oracle_result_copy_sampled(res, _ptr(out["ssupport"], ctypes.c_int64),
                                               _ptr(out["scount"], ctypes.c_int64))
                lib.oracle_result_copy_sampled_domains(res, _ptr(out["spop"], ctypes.c_int64),
                                                       _ptr(out["sdeg"], ctypes.c_double))
    finally:
        lib.oracle_free(res)
    return out


def pattern_support(g, labels, adj: int, mode: str = "edge", max_maps: int = 0) -> tuple[int, int]:
    """(MNI support, embedding count) of one pattern, by matching every label-preserving
    monomorphism (edge-induced) or induced embedding (vertex-induced) of it.  Raises
    OverflowError when more than max_maps maps exist (max_maps > 0)."""
    lib = _load()
    k = len(labels)
    row_ptr = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    lab = np.ascontiguousarray(g.labels, dtype=np.int32)
    plab = np.ascontiguousarray(labels, dtype=np.int32)
    rows = np.zeros(max(k, 1), np.uint32)
    for i in range(k):
        for j in range(i + 1, k):
            if (int(adj) >> (i * k + j)) & 1:
                rows[i] |= np.uint32(1 << j)
                rows[j] |= np.uint32(1 << i)
    sup, cnt = ctypes.c_int64(), ctypes.c_int64()
    rc = lib.oracle_pattern_support_rows(g.n, _ptr(row_ptr, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                                         _ptr(lab, ctypes.c_int32), k, _ptr(plab, ctypes.c_int32),
                                         _ptr(rows, ctypes.c_uint32), MODES[mode], int(max_maps),
                                         ctypes.byref(sup), ctypes.byref(cnt))
    if rc == -2:
        raise OverflowError("pattern has more than max_maps maps")
    if rc != 0:
        raise ValueError("oracle_pattern_support rejected its arguments")
    return int(sup.value), int(cnt.value)


def dissect(adj_rows) -> int:
    """3-vertex part (bit mask over positions, which are the vertex ids) of the smallest-vertex-
    first dissection of a connected graph."""
    rows = np.ascontiguousarray(adj_rows, dtype=np.uint32)
    return int(_load().oracle_dissect(len(rows), _ptr(rows, ctypes.c_uint32)))


def pattern_edges(adj: int, k: int) -> list[tuple[int, int]]:
    """Canonical edge list (i < j) of an ``adj`` word."""
    return [(i, j) for i in range(k) for j in range(i + 1, k) if (int(adj) >> (i * k + j)) & 1]


def dissect_join(adj_rows) -> tuple[int, int]:
    """(3-vertex part as a bit mask, join vertex) of the dissection of a connected graph whose
    positions are its vertex ids; (0, -1) when none exists."""
    rows = np.ascontiguousarray(adj_rows, dtype=np.uint32)
    j = ctypes.c_int32()
    m = int(_load().oracle_dissect_join(len(rows), _ptr(rows, ctypes.c_uint32), ctypes.byref(j)))
    return m, int(j.value)


def edge_kept(seed: int, p: float, x: int, y: int) -> bool:
    """Sampled mining's rule for one directed edge x -> y at rate p (kept at rate sqrt(p))."""
    return bool(_load().oracle_edge_kept(int(seed) & ((1 << 64) - 1), float(p), int(x), int(y)))


def kept(u, adj_rows, seed: int, p: float) -> bool:
    """Whether sampled mining at rate p keeps the embedding with ascending vertex ids u and
    adjacency rows over positions (k >= 3)."""
    uu = np.ascontiguousarray(u, dtype=np.int32)
    rows = np.ascontiguousarray(adj_rows, dtype=np.uint32)
    r = _load().oracle_kept(len(uu), _ptr(uu, ctypes.c_int32), _ptr(rows, ctypes.c_uint32),
                            int(seed) & ((1 << 64) - 1), float(p))
    if r < 0:
        raise ValueError("kept needs 3 <= k <= 9")
    return bool(r)


def mine_quota(g, k: int, t: int, mode: str = "edge", seed: int = 0, join_quota: int = 0,
               match_quota: int = 0) -> dict:
    """Patterns of exactly k vertices (3 <= k <= 9) whose MNI support over the embeddings drawn
    under Section 5's sampling quotas reaches t, by the method's own level-wise steps: size-3
    matching with at most ``match_quota`` candidate pieces per vertex, then joins l -> l+2 with at
    most ``join_quota``^2 candidate pieces per key group and, joining edges, ``join_quota`` edges
    per key vertex (0 = all).  Quotas 0 give exact mining.  Same dict layout as ``mine``."""
    lib = _load()
    row_ptr = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    labels = np.ascontiguousarray(g.labels, dtype=np.int32)
    res = lib.oracle_mine_quota(g.n, _ptr(row_ptr, ctypes.c_int32), _ptr(col, ctypes.c_int32),
                                _ptr(labels, ctypes.c_int32), k, MODES[mode], int(t), int(seed) & ((1 << 64) - 1),
                                int(join_quota), int(match_quota))
    if not res:
        raise ValueError("oracle_mine_quota rejected its arguments")
    try:
        out = _result(lib, res, k)
    finally:
        lib.oracle_free(res)
    return out


def quota_draw(h: int, c: int) -> tuple[int, int]:
    """(a, b) of the quota draw for hash h and modulus c >= 2: candidates (a j + b) mod c."""
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _load().oracle_quota_draw(int(h) & ((1 << 64) - 1), int(c), ctypes.byref(a), ctypes.byref(b))
    return int(a.value), int(b.value)
