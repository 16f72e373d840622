"""Second, independent oracle for tiny graphs: MNI support straight from its definition.

TEST INFRASTRUCTURE ONLY (imported by the test suite).

Definition 2 (paper Section 2.2) says sigma(P) = min over pattern vertices v of
|{f_i(v)}|, the f_i being P's embeddings.  Here every pattern candidate P is a labeled graph on
positions 0..k-1 and f ranges over *every injective map* [k] -> V(G) that is

  * a monomorphism (labels equal, each pattern edge maps to a graph edge) -- edge-induced; or
  * an induced embedding (labels equal, pattern edge <=> graph edge)     -- vertex-induced.

Candidates are all connected labeled graphs on k positions, grouped into isomorphism classes by
an explicit search over bijections (Definition 1, label-preserving).  The number of embeddings
(subgraphs, not maps) of a class is #maps / |Aut(P)|.  Nothing here uses a canonical form, ESU
or any code of the C oracle; cost grows like n^k, so keep n <= 8 and k <= 5.
"""
from __future__ import annotations

import itertools

import numpy as np


def _connected(k: int, edges) -> bool:
    adj = {i: set() for i in range(k)}
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    seen, stack = {0}, [0]
    while stack:
        x = stack.pop()
        for y in adj[x]:
            if y not in seen:
                seen.add(y)
                stack.append(y)
    return len(seen) == k


def isomorphic(k, la, ea, lb, eb) -> bool:
    """Label-preserving isomorphism between (la, ea) and (lb, eb) on k positions."""
    if sorted(la) != sorted(lb) or len(ea) != len(eb):
        return False
    sa = {frozenset(e) for e in ea}
    sb = {frozenset(e) for e in eb}
    for f in itertools.permutations(range(k)):
        if any(la[i] != lb[f[i]] for i in range(k)):
            continue
        if all(frozenset((f[a], f[b])) in sb for a, b in sa):
            return True
    return False


def automorphisms(k, lab, edges) -> int:
    s = {frozenset(e) for e in edges}
    n = 0
    for f in itertools.permutations(range(k)):
        if any(lab[i] != lab[f[i]] for i in range(k)):
            continue
        if all(frozenset((f[a], f[b])) in s for a, b in s):
            n += 1
    return n


def pattern_classes(k: int, label_set) -> list[tuple[tuple, tuple]]:
    """One representative (labels, edges) per isomorphism class of connected labeled graphs."""
    pairs = [(i, j) for i in range(k) for j in range(i + 1, k)]
    reps = []
    buckets: dict = {}
    for mask in range(1 << len(pairs)):
        edges = tuple(p for q, p in enumerate(pairs) if mask >> q & 1)
        if len(edges) < k - 1 or not _connected(k, edges):
            continue
        deg = [0] * k
        for a, b in edges:
            deg[a] += 1
            deg[b] += 1
        for lab in itertools.product(sorted(label_set), repeat=k):
            inv = (len(edges), tuple(sorted(zip(lab, deg))))
            bucket = buckets.setdefault(inv, [])
            if any(isomorphic(k, lab, edges, rl, re) for rl, re in bucket):
                continue
            bucket.append((lab, edges))
            reps.append((lab, edges))
    return reps


def mine(g, k: int, t: int, mode: str = "edge") -> list[dict]:
    """Every k-vertex pattern with support >= t, as dicts {labels, edges, support, count}."""
    n = g.n
    nbr = [set(g.col[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(n)]
    lab_g = g.labels.tolist()
    out = []
    for lab, edges in pattern_classes(k, set(lab_g)):
        non_edges = [(i, j) for i in range(k) for j in range(i + 1, k) if (i, j) not in set(edges)]
        dom = [set() for _ in range(k)]
        maps = 0
        for f in itertools.permutations(range(n), k):
            if any(lab_g[f[i]] != lab[i] for i in range(k)):
                continue
            if not all(f[b] in nbr[f[a]] for a, b in edges):
                continue
            if mode == "vertex" and any(f[b] in nbr[f[a]] for a, b in non_edges):
                continue
            maps += 1
            for i in range(k):
                dom[i].add(f[i])
        if maps == 0:
            continue
        sigma = min(len(d) for d in dom)
        if sigma >= t:
            out.append({"labels": lab, "edges": edges, "support": sigma,
                        "count": maps // automorphisms(k, lab, edges)})
    return out


def same_patterns(k: int, brute: list[dict], oracle: dict) -> tuple[bool, str]:
    """Match brute-force classes to oracle rows by explicit isomorphism; compare support and
    embedding count."""
    if len(brute) != len(oracle["support"]):
        return False, f"pattern count {len(brute)} (brute) != {len(oracle['support'])} (oracle)"
    used = set()
    for q in range(len(oracle["support"])):
        lab = tuple(int(x) for x in oracle["labels"][q])
        adj = int(oracle["adj"][q])
        edges = [(i, j) for i in range(k) for j in range(i + 1, k) if adj >> (i * k + j) & 1]
        hit = None
        for b, row in enumerate(brute):
            if b not in used and isomorphic(k, lab, edges, row["labels"], row["edges"]):
                hit = b
                break
        if hit is None:
            return False, f"oracle pattern {lab} {edges} has no brute-force class"
        used.add(hit)
        row = brute[hit]
        if row["support"] != int(oracle["support"][q]) or row["count"] != int(oracle["count"][q]):
            return False, (f"pattern {lab} {edges}: brute (sigma={row['support']}, count={row['count']}) "
                           f"!= oracle (sigma={int(oracle['support'][q])}, count={int(oracle['count'][q])})")
    return True, "ok"
