"""Pins for the CPU oracle at k = 9 (Section 6, Table 3 mines 9-vertex patterns), no GPU.

Closed forms of complete graphs, paths, cycles and stars; agreement of the two independent parts
of the oracle (ESU enumeration with canonical codes, and the backtracking matcher over
label-preserving maps); embedding totals against connected vertex sets and connected spanning
edge subsets counted by brute force here; minimality of the canonical code over all 9!
orders; anti-monotonicity; and exact mining by the quota oracle's level-wise steps."""
import itertools
import math

import numpy as np
import pytest

import graphgen as gg
import oracle
import oracle.brute as brute

K = 9


def _edges_of(g):
    return [(v, int(w)) for v in range(g.n) for w in g.col[g.row_ptr[v]:g.row_ptr[v + 1]] if v < w]


def _n_edges(adj):
    return len(oracle.pattern_edges(adj, K))


def test_adj_words_are_python_ints():
    o = oracle.mine(gg.complete(K), K, 1, "vertex")
    assert o["adj"].dtype == object
    assert int(o["adj"][0]) == sum(1 << (i * K + j) for i in range(K) for j in range(i + 1, K))
    assert int(o["adj"][0]).bit_length() > 64


@pytest.mark.parametrize("n", [9, 10])
def test_complete_graph_vertex_induced(n):
    o = oracle.mine(gg.complete(n), K, 1, "vertex")
    assert len(o["support"]) == 1 and o["support"][0] == n and o["count"][0] == math.comb(n, K)
    assert _n_edges(o["adj"][0]) == K * (K - 1) // 2


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_path(mode):
    n = 2 * K + 1
    o = oracle.mine(gg.path(n), K, 1, mode)
    assert len(o["support"]) == 1
    assert o["support"][0] == n - 2 * ((K - 1) // 2) and o["count"][0] == n - K + 1
    assert _n_edges(o["adj"][0]) == K - 1


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_cycle_longer_than_pattern(mode):
    n = K + 3
    o = oracle.mine(gg.cycle(n), K, 1, mode)
    assert len(o["support"]) == 1 and o["support"][0] == n and o["count"][0] == n
    assert _n_edges(o["adj"][0]) == K - 1


def test_cycle_whole():
    ov = oracle.mine(gg.cycle(K), K, 1, "vertex")
    assert len(ov["support"]) == 1 and ov["support"][0] == K and ov["count"][0] == 1
    oe = oracle.mine(gg.cycle(K), K, 1, "edge")
    assert {_n_edges(a): int(c) for a, c in zip(oe["adj"], oe["count"])} == {K: 1, K - 1: K}
    assert np.all(oe["support"] == K)


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_star(mode):
    leaves = 10
    o = oracle.mine(gg.star(leaves), K, 1, mode)
    assert len(o["support"]) == 1 and o["support"][0] == 1
    assert o["count"][0] == math.comb(leaves, K - 1)


def test_matcher_closed_forms():
    adj = sum(1 << (i * K + i + 1) for i in range(K - 1))      # the path P_9
    assert oracle.pattern_support(gg.path(12), [0] * K, adj) == (12 - 2 * 4, 4)
    assert oracle.pattern_support(gg.cycle(11), [0] * K, adj) == (11, 11)
    assert oracle.pattern_support(gg.path(8), [0] * K, adj) == (0, 0)


@pytest.mark.parametrize("mode", ["edge", "vertex"])
@pytest.mark.parametrize("seed", [0, 1])
def test_matcher_agrees_with_enumeration(mode, seed):
    g = gg.tree_plus(12, 3, 3, seed)
    o = oracle.mine(g, K, 1, mode)
    assert len(o["support"]) > 5
    for lab, adj, s, c in zip(o["labels"], o["adj"], o["support"], o["count"]):
        assert oracle.pattern_support(g, lab, int(adj), mode) == (int(s), int(c))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_embedding_totals_by_brute_force(seed):
    """Vertex-induced: one embedding per connected 9-vertex set; edge-induced: one per connected
    spanning edge subset of such a set."""
    g = gg.tree_plus(12, 3, 2, seed)
    edges = _edges_of(g)
    n_sets = n_subsets = 0
    for vs in itertools.combinations(range(g.n), K):
        idx = {v: i for i, v in enumerate(vs)}
        ind = [(idx[a], idx[b]) for a, b in edges if a in idx and b in idx]
        if not brute._connected(K, ind):
            continue
        n_sets += 1
        for r in range(K - 1, len(ind) + 1):
            n_subsets += sum(1 for sub in itertools.combinations(ind, r) if brute._connected(K, list(sub)))
    assert n_sets > 10
    assert int(oracle.mine(g, K, 1, "vertex")["count"].sum()) == n_sets
    assert int(oracle.mine(g, K, 1, "edge")["count"].sum()) == n_subsets


def test_canonical_code_is_minimal():
    g = gg.tree_plus(11, 2, 2, 3)
    o = oracle.mine(g, K, 1, "vertex")
    pairs = [(i, j) for i in range(K) for j in range(i + 1, K)]
    for q in (0, len(o["support"]) - 1):
        lab = [int(x) for x in o["labels"][q]]
        es = {frozenset(e) for e in oracle.pattern_edges(o["adj"][q], K)}
        mine = (lab, [1 if frozenset(p) in es else 0 for p in pairs])
        for perm in itertools.permutations(range(K)):
            cl = [lab[perm[c]] for c in range(K)]
            if cl > lab:
                continue
            ca = [1 if frozenset((perm[a], perm[b])) in es else 0 for a, b in pairs]
            assert (cl, ca) >= mine


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_anti_monotone(mode):
    g = gg.tree_plus(12, 3, 2, 5)
    big = oracle.mine(g, K, 1, mode)
    small = oracle.mine(g, K - 1, 1, mode)
    sup = {(tuple(int(x) for x in l), int(a)): int(s) for l, a, s in zip(small["labels"], small["adj"], small["support"])}
    checked = 0
    for lab, adj, sig in zip(big["labels"], big["adj"], big["support"]):
        lab = [int(x) for x in lab]
        edges = oracle.pattern_edges(adj, K)
        for drop in range(K):
            keep = [v for v in range(K) if v != drop]
            sub = [(keep.index(a), keep.index(b)) for a, b in edges if drop not in (a, b)]
            if not brute._connected(K - 1, sub):
                continue
            sg = gg.from_edges(K - 1, sub, np.array([lab[v] for v in keep], np.int32), 2)
            c = oracle.mine(sg, K - 1, 1, "vertex")
            key = (tuple(int(x) for x in c["labels"][0]), int(c["adj"][0]))
            assert sig <= sup[key]
            checked += 1
    assert checked > 10


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_quota_oracle_without_quotas_is_exact(mode):
    g = gg.tree_plus(13, 3, 2, 7)
    for t in (1, 2):
        a = oracle.mine(g, K, t, mode)
        b = oracle.mine_quota(g, K, t, mode, seed=0, join_quota=0, match_quota=0)
        for key in ("labels", "adj", "support", "count"):
            assert np.array_equal(a[key], b[key]), (t, key)


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_quota_supports_are_lower_bounds(mode):
    """Section 5's quotas draw a subset of the embeddings: every pattern they report is truly
    frequent, with a support and count no larger than the exact ones."""
    g = gg.tree_plus(14, 4, 2, 3)
    exact = oracle.mine(g, K, 1, mode)
    ex = {(tuple(int(x) for x in l), int(a)): (int(s), int(c))
          for l, a, s, c in zip(exact["labels"], exact["adj"], exact["support"], exact["count"])}
    checked = 0
    for x in (2, 3):
        q = oracle.mine_quota(g, K, 1, mode, seed=7, join_quota=x)
        for l, a, s, c in zip(q["labels"], q["adj"], q["support"], q["count"]):
            key = (tuple(int(v) for v in l), int(a))
            assert key in ex and int(s) <= ex[key][0] and int(c) <= ex[key][1]
            checked += 1
    assert checked > 0
