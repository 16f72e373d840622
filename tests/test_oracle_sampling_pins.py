"""Pins for the oracle's dissection (Section 4.3, Algorithm 1) and its sampling rule (Section 5,
read as a counter-based rate), each checked against something other than the oracle itself:

* the worked example of Section 4.3 (``tests/golden/dissect_example.txt``);
* the closed form of the four-vertex dissection (the greedy round from the smallest vertex
  always succeeds there, so the part is {m, n1, n2} and the join its smallest vertex next to
  the fourth);
* validity and totality on every connected graph of at most six vertex ids, and, where the
  greedy rule finds nothing, minimality among every valid dissection found by brute force;
* splitmix64 written here from its published definition (Steele, Lea and Flood 2014);
* the binomial law of the kept fraction of directed edges;
* the sampled supports and counts of whole mining runs against an independent enumeration of
  every embedding of graphs with at most eight vertices.
No GPU is used.
"""
import itertools
import math
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
import oracle.brute as brute

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1


# --------------------------------------------------------------------- helpers (independent)

def splitmix64(x: int) -> int:
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def edge_kept_ref(seed: int, p: float, x: int, y: int) -> bool:
    thr = int(math.sqrt(p) * 2.0 ** 64)
    h = splitmix64(seed & M64)
    h = splitmix64(h ^ (x & 0xFFFFFFFF))
    h = splitmix64(h ^ (y & 0xFFFFFFFF))
    return h < thr


def nbrs(rows, h):
    return {j for j in range(len(rows)) if rows[h] >> j & 1}


def connected_set(rows, vs):
    vs = set(vs)
    if not vs:
        return False
    start = min(vs)
    seen, stack = {start}, [start]
    while stack:
        x = stack.pop()
        for y in nbrs(rows, x) & vs:
            if y not in seen:
                seen.add(y)
                stack.append(y)
    return seen == vs


def valid_dissections(rows):
    """Every (sorted 3-part, join) whose part is connected and whose remainder plus the join
    is connected; positions are ids."""
    k = len(rows)
    out = []
    for part in itertools.combinations(range(k), 3):
        if not connected_set(rows, part):
            continue
        rest = set(range(k)) - set(part)
        for j in part:
            if connected_set(rows, rest | {j}):
                out.append((part, j))
    return out


def greedy_dissection(rows):
    """The greedy round of Section 4.3 from each start vertex in ascending id order; None when
    no start vertex gives a dissection."""
    k = len(rows)
    for start in range(k):
        vis = {start}
        for _ in range(2):
            cand = set().union(*(nbrs(rows, h) for h in vis)) - vis
            if not cand:
                break
            vis.add(min(cand))
        if len(vis) < 3:
            continue
        rest = set(range(k)) - vis
        for j in sorted(vis):
            if connected_set(rows, rest | {j}):
                return tuple(sorted(vis)), j
    return None


def all_connected_graphs(k):
    pairs = [(i, j) for i in range(k) for j in range(i + 1, k)]
    for mask in range(1 << len(pairs)):
        rows = [0] * k
        for q, (a, b) in enumerate(pairs):
            if mask >> q & 1:
                rows[a] |= 1 << b
                rows[b] |= 1 << a
        if connected_set(rows, range(k)):
            yield rows


def mask_to_part(m):
    return tuple(h for h in range(32) if m >> h & 1)


# --------------------------------------------------------------------- dissection pins

def _golden_cases():
    cases = []
    for line in open(os.path.join(GOLDEN, "dissect_example.txt")):
        if line.startswith("case"):
            parts = [p.strip() for p in line[4:].split("|")]
            verts = [int(x) for x in parts[0].split()]
            edges = [tuple(int(y) for y in e.split("-")) for e in parts[1].split()]
            cases.append((verts, edges, [int(x) for x in parts[2].split()], int(parts[3])))
    return cases


@pytest.mark.parametrize("case", _golden_cases())
def test_oracle_dissect_paper_example(case):
    """Section 4.3's worked example: 34257 dissects into {2,3,4} + {3,5,7} joined at 3, and
    37485 into {3,4,5} + {3,8,7}, so the join of 374 with 385 is dropped."""
    verts, edges, l_exp, join_exp = case
    order = sorted(verts)              # the oracle's positions are ascending ids
    idx = {v: i for i, v in enumerate(order)}
    rows = [0] * len(order)
    for a, b in edges:
        rows[idx[a]] |= 1 << idx[b]
        rows[idx[b]] |= 1 << idx[a]
    m, j = oracle.dissect_join(rows)
    assert sorted(order[h] for h in mask_to_part(m)) == l_exp
    assert order[j] == join_exp


def test_oracle_dissect_four_vertex_closed_form():
    """k = 4: the part is {m, n1, n2} (m = 0, the smallest id; n1 its smallest neighbour; n2 the
    smallest further neighbour of {m, n1}) and the join is the smallest part vertex adjacent to
    the fourth vertex.  The fourth vertex is always adjacent to the part (the graph is
    connected), so this answer exists for every graph."""
    n = 0
    for rows in all_connected_graphs(4):
        n1 = min(nbrs(rows, 0))
        n2 = min((nbrs(rows, 0) | nbrs(rows, n1)) - {0, n1})
        part = {0, n1, n2}
        (fourth,) = set(range(4)) - part
        join = min(nbrs(rows, fourth) & part)
        m, j = oracle.dissect_join(rows)
        assert set(mask_to_part(m)) == part and j == join, rows
        n += 1
    assert n == 38   # connected labeled graphs on 4 vertices (OEIS A001187)


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_oracle_dissect_total_valid_and_minimal(k):
    """Theorem 1 on every connected graph of k ids: a dissection exists, and the oracle returns
    a valid one -- the greedy one when the greedy round finds any, otherwise the smallest
    (sorted part, join) of every valid dissection listed by brute force."""
    graphs = fallbacks = 0
    for rows in all_connected_graphs(k):
        graphs += 1
        m, j = oracle.dissect_join(rows)
        part = mask_to_part(m)
        valid = valid_dissections(rows)
        assert valid, rows
        assert (part, j) in valid, (rows, part, j)
        g = greedy_dissection(rows)
        if g is not None:
            assert (part, j) == g, (rows, part, j, g)
        else:
            fallbacks += 1
            assert (part, j) == min(valid), (rows, part, j)
    assert graphs == {3: 4, 4: 38, 5: 728, 6: 26704}[k]   # A001187
    if k < 6:
        assert fallbacks == 0   # the greedy rule always answers below six vertices


def test_oracle_dissect_needs_fallback_at_six():
    """Theorem 1 promises a dissection, not that the greedy round finds one: 32 of the 26704
    connected graphs on six ids have none, and there the exhaustive rule answers."""
    hits = sum(1 for rows in all_connected_graphs(6) if greedy_dissection(rows) is None)
    assert hits == 32


# --------------------------------------------------------------------- sampling rule pins

def test_edge_kept_is_published_splitmix():
    rng = np.random.default_rng(3)
    for _ in range(400):
        seed = int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2))
        x, y = (int(v) for v in rng.integers(0, 2 ** 31, size=2))
        p = float(rng.choice([0.01, 0.05, 0.25, 0.5, 0.9]))
        assert oracle.edge_kept(seed, p, x, y) == edge_kept_ref(seed, p, x, y), (seed, p, x, y)


@pytest.mark.parametrize("p", [0.01, 0.05, 0.25])
def test_kept_edge_fraction_is_binomial(p):
    """Each directed edge is kept independently at rate q = sqrt(p): over E edges the kept
    count lies within five standard deviations of E q."""
    g = gg.workload("cl100k", scale=0.02, cap=60)
    src = np.repeat(np.arange(g.n), g.degrees())
    E = len(g.col)
    kept = sum(oracle.edge_kept(11, p, int(a), int(b)) for a, b in zip(src, g.col))
    q = math.sqrt(p)
    assert abs(kept - E * q) <= 5 * math.sqrt(E * q * (1 - q)), (kept, E, q)


@pytest.mark.parametrize("k", [3, 4])
def test_kept_embedding_fraction_is_p(k):
    """An embedding is kept when two distinct directed edges are, so the kept fraction of all
    embeddings is p in expectation (checked within 15 % at p = 0.25)."""
    g = gg.workload("er1000", scale=0.5)
    o = oracle.mine(g, k, 1, sample=(0.25, 5))
    frac = o["scount"].sum() / o["count"].sum()
    assert abs(frac / 0.25 - 1) < 0.15, frac


def _embeddings(g, k, mode):
    """Every embedding of g as (ascending ids, adjacency rows over positions)."""
    nb = [set(g.col[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]
    for vs in itertools.combinations(range(g.n), k):
        pairs = [(a, b) for a in range(k) for b in range(a + 1, k) if vs[b] in nb[vs[a]]]
        subsets = [pairs] if mode == "vertex" else (
            [e for q, e in enumerate(pairs) if mask >> q & 1] for mask in range(1, 1 << len(pairs)))
        for es in subsets:
            rows = [0] * k
            for a, b in es:
                rows[a] |= 1 << b
                rows[b] |= 1 << a
            if connected_set(rows, range(k)):
                yield vs, rows


def _kept_ref(vs, rows, seed, p):
    """The sampling rule from Section 5's reading: the 3-vertex part of the embedding's
    dissection, seen from its join vertex j, must be made of kept directed edges -- j -> x and
    j -> y when j is next to both other part vertices, else j -> c and c -> z along the wedge
    centred at c."""
    part, j = greedy_dissection(rows) or min(valid_dissections(rows))
    x, y = (h for h in part if h != j)
    ax, ay = bool(rows[j] >> x & 1), bool(rows[j] >> y & 1)
    if ax and ay:
        return edge_kept_ref(seed, p, vs[j], vs[x]) and edge_kept_ref(seed, p, vs[j], vs[y])
    c, z = (x, y) if ax else (y, x)
    return edge_kept_ref(seed, p, vs[j], vs[c]) and edge_kept_ref(seed, p, vs[c], vs[z])


@pytest.mark.parametrize("mode", ["edge", "vertex"])
@pytest.mark.parametrize("k,seed", [(3, 1), (4, 2), (4, 7), (5, 3)])
def test_sampled_statistics_match_independent_count(mode, k, seed):
    """Sampled mining statistics of the oracle (kept embeddings and MNI over their images, per
    pattern) against a count made here: every embedding of a graph with 8 vertices, the rule
    above, and every label-preserving isomorphism from the oracle's pattern onto each kept
    embedding (Definition 2)."""
    g = gg.random_small(8, 0.5, 2, seed)
    p = 0.35
    o = oracle.mine(g, k, 1, mode, sample=(p, seed))
    lab_g = g.labels.tolist()
    pats = []
    for q in range(len(o["support"])):
        lab = [int(x) for x in o["labels"][q]]
        pats.append((lab, oracle.pattern_edges(o["adj"][q], k)))
    scount = [0] * len(pats)
    images = [[set() for _ in range(k)] for _ in pats]
    total = 0
    for vs, rows in _embeddings(g, k, mode):
        total += 1
        assert oracle.kept(list(vs), rows, seed, p) == _kept_ref(vs, rows, seed, p)
        if not _kept_ref(vs, rows, seed, p):
            continue
        elab = [lab_g[v] for v in vs]
        eedges = [(a, b) for a in range(k) for b in range(a + 1, k) if rows[a] >> b & 1]
        es = {frozenset(e) for e in eedges}
        hit = [q for q, (pl, pe) in enumerate(pats) if brute.isomorphic(k, pl, pe, elab, eedges)]
        assert len(hit) == 1
        q = hit[0]
        scount[q] += 1
        pl, pe = pats[q]
        for f in itertools.permutations(range(k)):   # pattern position c -> embedding position f[c]
            if all(pl[c] == elab[f[c]] for c in range(k)) and \
                    all(frozenset((f[a], f[b])) in es for a, b in pe):
                for c in range(k):
                    images[q][c].add(vs[f[c]])
    assert total == int(o["count"].sum())
    assert list(o["scount"]) == scount
    assert list(o["ssupport"]) == [min(len(s) for s in im) for im in images]
    deg = g.degrees()
    for q, im in enumerate(images):
        assert list(o["spop"][q]) == [len(s) for s in im]
        assert np.allclose(o["sdeg"][q], [sum(math.log1p(deg[v]) for v in s) for s in im], rtol=1e-12, atol=1e-12)
