"""Seeded synthetic labeled graphs, shared by the CUDA path's tests/bench and the CPU oracle.

This module draws graphs and labels and writes them as a simple undirected CSR.  It holds
none of the mining method's arithmetic (no enumeration, no patterns, no support): both the
GPU library and the oracle receive the same arrays from here.

Graph families (the paper's workloads are labeled sparse graphs, Section 6 / Table 1; the
real datasets are replaced by these stand-ins):

* ``erdos_renyi(n, avg_degree, seed)`` -- G(n, p) with p = avg_degree / (n - 1).
* ``chung_lu(n, m, beta, seed, cap)`` -- expected-degree power-law graph: weights
  w_i ~ i^(-1/(beta-1)), rescaled to sum 2m and clamped at ``cap`` (iterated), endpoints
  drawn i.i.d. proportional to w, self-loops and duplicate edges dropped, redrawn until m
  unique edges exist; vertex ids are then shuffled so hubs are not the lowest ids.
* small closed-form graphs (complete, path, cycle, star, complete bipartite, spider).

Labels: ``uniform_labels`` or ``zipf_labels`` (P(r) proportional to (r+1)^-s), drawn i.i.d.
and independent of degree.

CSR convention: ``row_ptr`` int32[n+1], ``col`` int32[2m] with every undirected edge stored
in both directions, each row sorted ascending, no self-loops, no duplicates.
"""
from __future__ import annotations

import hashlib
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Graph", "from_edges", "erdos_renyi", "chung_lu", "uniform_labels", "zipf_labels",
    "complete", "path", "cycle", "star", "complete_bipartite", "spider", "random_small",
    "relabel_vertices", "workload", "WORKLOADS",
]


@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray          # int32[n+1]
    col: np.ndarray              # int32[2m]
    labels: np.ndarray           # int32[n]
    num_labels: int
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.col.shape[0] // 2)

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def edges(self) -> np.ndarray:
        """Undirected edges (u < w) as int64[m, 2]."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        dst = self.col.astype(np.int64)
        keep = src < dst
        return np.stack([src[keep], dst[keep]], axis=1)

    def content_hash(self) -> str:
        h = hashlib.sha256()
        for a in (self.row_ptr, self.col, self.labels):
            h.update(np.ascontiguousarray(a).tobytes())
        h.update(str(self.num_labels).encode())
        return h.hexdigest()[:16]

    def stats(self) -> dict:
        d = self.degrees()
        out = {"n": self.n, "m": self.m, "d_max": int(d.max()) if self.n else 0,
               "d_mean": float(d.mean()) if self.n else 0.0}
        for r in (2, 3, 4):
            c = np.ones_like(d, dtype=np.float64)
            for j in range(r):
                c *= np.maximum(d - j, 0)
            fact = float(np.prod(np.arange(1, r + 1)))
            out[f"sum_C(d,{r})"] = float(c.sum() / fact)
        return out


def from_edges(n: int, edges, labels, num_labels: int | None = None, meta: dict | None = None) -> Graph:
    """Build a simple undirected CSR from an edge list (any orientation, duplicates and
    self-loops are dropped)."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    lo = np.minimum(e[:, 0], e[:, 1])
    hi = np.maximum(e[:, 0], e[:, 1])
    key = np.unique(lo * n + hi) if e.size else np.zeros(0, np.int64)
    lo, hi = key // n, key % n
    src = np.concatenate([lo, hi])
    dst = np.concatenate([hi, lo])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, src + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    labels = np.asarray(labels, dtype=np.int32).reshape(n)
    if num_labels is None:
        num_labels = int(labels.max()) + 1 if n else 1
    return Graph(n=n, row_ptr=row_ptr.astype(np.int32), col=dst.astype(np.int32),
                 labels=labels, num_labels=int(num_labels), meta=dict(meta or {}))


def uniform_labels(n: int, num_labels: int, rng: np.random.Generator) -> np.ndarray:
    return rng.integers(0, num_labels, size=n, dtype=np.int64).astype(np.int32)


def zipf_labels(n: int, num_labels: int, s: float, rng: np.random.Generator) -> np.ndarray:
    p = (np.arange(num_labels, dtype=np.float64) + 1.0) ** (-s)
    p /= p.sum()
    return rng.choice(num_labels, size=n, p=p).astype(np.int32)


def erdos_renyi(n: int, avg_degree: float, seed: int, num_labels: int = 1,
                label_law: str = "uniform", zipf_s: float = 1.0) -> Graph:
    """G(n, p), p = avg_degree/(n-1); labels drawn after the edges."""
    rng = np.random.default_rng(seed)
    p = avg_degree / max(n - 1, 1)
    iu, ju = np.triu_indices(n, k=1)
    keep = rng.random(iu.shape[0]) < p
    edges = np.stack([iu[keep], ju[keep]], axis=1)
    labels = _labels(n, num_labels, label_law, zipf_s, rng)
    return from_edges(n, edges, labels, num_labels,
                      meta={"family": "erdos_renyi", "n": n, "avg_degree": avg_degree, "seed": seed})


def _labels(n, num_labels, law, s, rng):
    if num_labels <= 1:
        return np.zeros(n, dtype=np.int32)
    if law == "uniform":
        return uniform_labels(n, num_labels, rng)
    if law == "zipf":
        return zipf_labels(n, num_labels, s, rng)
    raise ValueError(f"unknown label law {law!r}")


def chung_lu_weights(n: int, m: int, beta: float, cap: float | None) -> np.ndarray:
    w = np.arange(1, n + 1, dtype=np.float64) ** (-1.0 / (beta - 1.0))
    target = 2.0 * m
    for _ in range(100):
        w *= target / w.sum()
        if cap is None or w.max() <= cap * (1 + 1e-12):
            break
        w = np.minimum(w, cap)
    return w


def chung_lu(n: int, m: int, beta: float, seed: int, cap: float | None = None,
             num_labels: int = 1, label_law: str = "uniform", zipf_s: float = 1.0,
             shuffle_ids: bool = True) -> Graph:
    """Chung-Lu expected-degree graph with exactly m unique undirected edges."""
    rng = np.random.default_rng(seed)
    if cap is None:
        cap = float(np.sqrt(2.0 * m))
    w = chung_lu_weights(n, m, beta, cap)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    have = np.zeros(0, dtype=np.int64)
    need = m
    while need > 0:
        draw = int(need * 1.1) + 1024
        u = np.searchsorted(cdf, rng.random(draw), side="right")
        v = np.searchsorted(cdf, rng.random(draw), side="right")
        u = np.minimum(u, n - 1)
        v = np.minimum(v, n - 1)
        ok = u != v
        lo = np.minimum(u[ok], v[ok]).astype(np.int64)
        hi = np.maximum(u[ok], v[ok]).astype(np.int64)
        key = lo * n + hi
        # keep first occurrences in draw order so the result depends only on the seed
        _, first = np.unique(key, return_index=True)
        key = key[np.sort(first)]
        key = key[~np.isin(key, have)]
        key = key[:need]
        have = np.concatenate([have, key])
        need = m - have.shape[0]
    lo, hi = have // n, have % n
    if shuffle_ids:
        perm = rng.permutation(n)
        lo, hi = perm[lo], perm[hi]
    labels = _labels(n, num_labels, label_law, zipf_s, rng)
    return from_edges(n, np.stack([lo, hi], axis=1), labels, num_labels,
                      meta={"family": "chung_lu", "n": n, "m": m, "beta": beta, "seed": seed,
                            "cap": cap, "label_law": label_law, "zipf_s": zipf_s})


# ---------------------------------------------------------------- small closed-form graphs

def complete(n: int, labels=None) -> Graph:
    e = [(i, j) for i in range(n) for j in range(i + 1, n)]
    return from_edges(n, e, np.zeros(n, np.int32) if labels is None else labels)


def path(n: int, labels=None) -> Graph:
    e = [(i, i + 1) for i in range(n - 1)]
    return from_edges(n, e, np.zeros(n, np.int32) if labels is None else labels)


def cycle(n: int, labels=None) -> Graph:
    e = [(i, (i + 1) % n) for i in range(n)]
    return from_edges(n, e, np.zeros(n, np.int32) if labels is None else labels)


def star(leaves: int, labels=None) -> Graph:
    n = leaves + 1
    e = [(0, i) for i in range(1, n)]
    return from_edges(n, e, np.zeros(n, np.int32) if labels is None else labels)


def complete_bipartite(a: int, b: int) -> Graph:
    """K_{a,b}; side A gets label 0, side B label 1."""
    e = [(i, a + j) for i in range(a) for j in range(b)]
    labels = np.array([0] * a + [1] * b, dtype=np.int32)
    return from_edges(a + b, e, labels, 2)


def spider(prongs: int = 3, prong_len: int = 2) -> Graph:
    """A centre with ``prongs`` paths of ``prong_len`` vertices each."""
    e = []
    nxt = 1
    for _ in range(prongs):
        prev = 0
        for _ in range(prong_len):
            e.append((prev, nxt))
            prev = nxt
            nxt += 1
    return from_edges(nxt, e, np.zeros(nxt, np.int32))


def random_small(n: int, p: float, num_labels: int, seed: int) -> Graph:
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, k=1)
    keep = rng.random(iu.shape[0]) < p
    labels = rng.integers(0, num_labels, size=n).astype(np.int32)
    return from_edges(n, np.stack([iu[keep], ju[keep]], 1), labels, num_labels)


def tree_plus(n: int, extra: int, num_labels: int, seed: int) -> Graph:
    """A random labeled tree on n vertices (vertex v > 0 hangs off a uniform earlier vertex) plus
    `extra` further distinct edges: sparse and connected, so the connected 9-vertex subgraphs
    stay few enough for brute force."""
    rng = np.random.default_rng(seed)
    edges = set()
    for v in range(1, n):
        edges.add((int(rng.integers(v)), v))
    while len(edges) < n - 1 + extra:
        a, b = sorted(int(x) for x in rng.choice(n, 2, replace=False))
        edges.add((a, b))
    labels = rng.integers(num_labels, size=n).astype(np.int32)
    return from_edges(n, sorted(edges), labels, num_labels)


def relabel_vertices(g: Graph, perm: np.ndarray) -> Graph:
    """Same graph with vertex v renamed perm[v]."""
    perm = np.asarray(perm, dtype=np.int64)
    e = g.edges()
    labels = np.empty(g.n, dtype=np.int32)
    labels[perm] = g.labels
    return from_edges(g.n, perm[e], labels, g.num_labels, meta=dict(g.meta))


# ---------------------------------------------------------------- named workloads

# Degree caps are parameters of the Chung-Lu construction, given per call (``cap=``).  A cap
# changes the mining work by orders of magnitude, so every measurement records the one it used.
WORKLOADS = {
    # ER G(n=1000, avg degree 6), 4 uniform labels; k <= 3 at t = 30.
    "er1000": dict(family="er", n=1000, avg_degree=6.0, seed=0, num_labels=4, label_law="uniform"),
    # MiCo-shaped: Chung-Lu 100k vertices, 1.1M edges, beta 2.1, 29 Zipf(1.2) labels.
    "cl100k": dict(family="cl", n=100_000, m=1_100_000, beta=2.1, seed=1, num_labels=29,
                   label_law="zipf", zipf_s=1.2, cap=None),
    # Chung-Lu 3.7M vertices, 16.5M edges, beta 2.3, 37 Zipf(1.0) labels.
    "cl3700k": dict(family="cl", n=3_700_000, m=16_500_000, beta=2.3, seed=2, num_labels=37,
                    label_law="zipf", zipf_s=1.0, cap=None),
    # CiteSeer-shaped: Chung-Lu 3312 vertices, 4732 edges, beta 2.5, degree cap 99, 6 uniform
    # labels (the shape of the citation graph the 9-vertex experiments of Section 6 use).
    "ci3k": dict(family="cl", n=3312, m=4732, beta=2.5, seed=4, num_labels=6, label_law="uniform", cap=99),
    # Chung-Lu 1.1M vertices, 3M edges, beta 2.0, 16 uniform labels.
    "cl1100k": dict(family="cl", n=1_100_000, m=3_000_000, beta=2.0, seed=3, num_labels=16,
                    label_law="uniform", cap=None),
}


def workload(name: str, scale: float = 1.0, cap: float | None | str = "default", seed: int | None = None) -> Graph:
    """Named workload graph.  ``scale`` shrinks n and m together (same beta, labels, mean
    degree) for small parity cases; ``cap`` overrides the Chung-Lu degree cap."""
    spec = dict(WORKLOADS[name])
    fam = spec.pop("family")
    if seed is not None:
        spec["seed"] = seed
    if fam == "er":
        n = max(8, int(round(spec["n"] * scale)))
        return erdos_renyi(n, spec["avg_degree"], spec["seed"], spec["num_labels"], spec["label_law"])
    n = max(16, int(round(spec["n"] * scale)))
    m = max(16, int(round(spec["m"] * scale)))
    c = spec.pop("cap")
    if cap != "default":
        c = cap
    return chung_lu(n, m, spec["beta"], spec["seed"], cap=c, num_labels=spec["num_labels"],
                    label_law=spec["label_law"], zipf_s=spec.get("zipf_s", 1.0))
