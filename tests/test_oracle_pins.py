"""Pins for the CPU oracle: brute force, closed forms, invariants (no GPU).

Each test checks the oracle against something other than itself: the injective-map brute
force of ``oracle/brute.py`` (Definition 2 taken literally), closed forms of complete graphs,
paths, cycles, stars and bipartite graphs, counts of connected graphs from the literature, and
invariants (vertex renaming, anti-monotonicity of MNI, minimality of the canonical code).
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


def _connected_counts():
    rows = {}
    with open(os.path.join(GOLDEN, "connected_graphs.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, unl, lab = (int(x) for x in line.split())
            rows[k] = (unl, lab)
    return rows


# --------------------------------------------------------------------- brute force

@pytest.mark.parametrize("mode", ["edge", "vertex"])
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_brute_force_labeled(mode, seed):
    g = gg.random_small(7, 0.45, 2, seed)
    for k in (1, 2, 3, 4):
        o = oracle.mine(g, k, 1, mode)
        ok, msg = brute.same_patterns(k, brute.mine(g, k, 1, mode), o)
        assert ok, f"k={k}: {msg}"


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_brute_force_unlabeled_k5(mode):
    g = gg.random_small(7, 0.5, 1, 11)
    o = oracle.mine(g, 5, 1, mode)
    ok, msg = brute.same_patterns(5, brute.mine(g, 5, 1, mode), o)
    assert ok, msg


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_brute_force_threshold(mode):
    g = gg.random_small(8, 0.4, 3, 5)
    for t in (1, 2, 3, 4):
        o = oracle.mine(g, 3, t, mode)
        ok, msg = brute.same_patterns(3, brute.mine(g, 3, t, mode), o)
        assert ok, f"t={t}: {msg}"


# --------------------------------------------------------------------- closed forms

@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_complete_graph_vertex_induced(k):
    n = k + 1
    o = oracle.mine(gg.complete(n), k, 1, "vertex")
    assert len(o["support"]) == 1
    assert o["support"][0] == n
    assert o["count"][0] == math.comb(n, k)
    assert int(o["adj"][0]) == sum(1 << (i * k + j) for i in range(k) for j in range(i + 1, k))


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_complete_graph_edge_induced_counts(k):
    unl, lab = _connected_counts()[k]
    n = k + 1 if k <= 5 else k
    o = oracle.mine(gg.complete(n), k, 1, "edge")
    assert len(o["support"]) == unl
    assert np.all(o["support"] == n)
    assert int(o["count"].sum()) == math.comb(n, k) * lab


@pytest.mark.parametrize("mode", ["edge", "vertex"])
@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_path(mode, k):
    n = 2 * k + 1
    o = oracle.mine(gg.path(n), k, 1, mode)
    assert len(o["support"]) == 1
    assert o["support"][0] == n - 2 * ((k - 1) // 2)
    assert o["count"][0] == n - k + 1
    assert len(oracle.pattern_edges(o["adj"][0], k)) == k - 1


def test_path_mni_counts_every_automorphic_image():
    # P_4, k = 2: the single edge pattern has both endpoints in one orbit, so sigma = 4 (all
    # vertices), not 3 as a single-map reading would give.
    o = oracle.mine(gg.path(4), 2, 1)
    assert list(o["support"]) == [4]


@pytest.mark.parametrize("mode", ["edge", "vertex"])
@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_cycle_longer_than_pattern(mode, k):
    n = k + 3
    o = oracle.mine(gg.cycle(n), k, 1, mode)
    assert len(o["support"]) == 1
    assert o["support"][0] == n and o["count"][0] == n
    assert len(oracle.pattern_edges(o["adj"][0], k)) == k - 1


@pytest.mark.parametrize("n", [4, 5, 6])
def test_cycle_whole(n):
    ov = oracle.mine(gg.cycle(n), n, 1, "vertex")
    assert len(ov["support"]) == 1 and ov["support"][0] == n and ov["count"][0] == 1
    assert len(oracle.pattern_edges(ov["adj"][0], n)) == n
    oe = oracle.mine(gg.cycle(n), n, 1, "edge")
    assert sorted(len(oracle.pattern_edges(a, n)) for a in oe["adj"]) == [n - 1, n]
    assert np.all(oe["support"] == n)
    by_edges = {len(oracle.pattern_edges(a, n)): int(c) for a, c in zip(oe["adj"], oe["count"])}
    assert by_edges == {n: 1, n - 1: n}


@pytest.mark.parametrize("mode", ["edge", "vertex"])
@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_star(mode, k):
    leaves = 6
    o = oracle.mine(gg.star(leaves), k, 1, mode)
    assert len(o["support"]) == 1
    # k=2: the edge's two ends share an orbit, so every vertex is an image; k>2: the centre has
    # exactly one image
    assert o["support"][0] == (leaves + 1 if k == 2 else 1)
    assert o["count"][0] == math.comb(leaves, k - 1)


@pytest.mark.parametrize("a,b", [(2, 3), (3, 5), (4, 4)])
def test_two_coloured_bipartite(a, b):
    o = oracle.mine(gg.complete_bipartite(a, b), 2, 1)
    assert len(o["support"]) == 1
    assert o["support"][0] == min(a, b)
    assert list(o["labels"][0]) == [0, 1]
    assert o["count"][0] == a * b


def test_threshold_is_inclusive():
    g = gg.path(5)
    assert len(oracle.mine(g, 2, 5)["support"]) == 1
    assert len(oracle.mine(g, 2, 6)["support"]) == 0


# --------------------------------------------------------------------- invariants

@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_vertex_renaming_invariance(mode):
    g = gg.workload("er1000", scale=0.1)
    rng = np.random.default_rng(7)
    h = gg.relabel_vertices(g, rng.permutation(g.n))
    for k in (2, 3, 4):
        a, b = oracle.mine(g, k, 1, mode), oracle.mine(h, k, 1, mode)
        for key in ("labels", "adj", "support", "count"):
            assert np.array_equal(a[key], b[key]), (k, key)


def _pattern_graph(lab, edges):
    return gg.from_edges(len(lab), edges, np.array(lab, np.int32), max(lab) + 1)


def _canon(lab, edges):
    """Canonical code of a connected labeled graph: mine the graph itself (vertex-induced, k = n)."""
    o = oracle.mine(_pattern_graph(lab, edges), len(lab), 1, "vertex")
    assert len(o["support"]) == 1
    return tuple(int(x) for x in o["labels"][0]), int(o["adj"][0])


def test_canonical_code_is_minimal_and_idempotent():
    g = gg.random_small(8, 0.45, 2, 21)
    k = 4
    o = oracle.mine(g, k, 1, "edge")
    pairs = [(i, j) for i in range(k) for j in range(i + 1, k)]
    for lab, adj in zip(o["labels"], o["adj"]):
        lab = [int(x) for x in lab]
        edges = oracle.pattern_edges(adj, k)
        assert _canon(lab, edges) == (tuple(lab), int(adj))
        es = {frozenset(e) for e in edges}
        mine = (lab, [1 if frozenset(p) in es else 0 for p in pairs])
        for perm in itertools.permutations(range(k)):
            cl = [lab[perm[c]] for c in range(k)]
            ca = [1 if frozenset((perm[a], perm[b])) in es else 0 for a, b in pairs]
            assert (cl, ca) >= mine


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_anti_monotone(mode):
    """sigma(P) <= sigma(P') for every connected sub-pattern P' obtained by deleting one
    vertex (and, edge-induced, one edge)."""
    g = gg.random_small(9, 0.4, 2, 4)
    k = 4
    big = oracle.mine(g, k, 1, mode)
    small = oracle.mine(g, k - 1, 1, mode)
    same = big
    sup_small = {(tuple(int(x) for x in l), int(a)): int(s)
                 for l, a, s in zip(small["labels"], small["adj"], small["support"])}
    sup_same = {(tuple(int(x) for x in l), int(a)): int(s)
                for l, a, s in zip(same["labels"], same["adj"], same["support"])}
    checked = 0
    for lab, adj, sig in zip(big["labels"], big["adj"], big["support"]):
        lab = [int(x) for x in lab]
        edges = oracle.pattern_edges(adj, k)
        for drop in range(k):
            keep = [v for v in range(k) if v != drop]
            sub_e = [(keep.index(a), keep.index(b)) for a, b in edges if drop not in (a, b)]
            sl = [lab[v] for v in keep]
            if not brute._connected(k - 1, sub_e):
                continue
            assert sig <= sup_small[_canon(sl, sub_e)]
            checked += 1
        if mode == "edge":
            for e in edges:
                rest = [x for x in edges if x != e]
                if brute._connected(k, rest):
                    assert sig <= sup_same[_canon(lab, rest)]
                    checked += 1
    assert checked > 10


def test_root_range_partitions_counts():
    """Enumeration by smallest vertex: disjoint root ranges partition the embedding counts."""
    g = gg.workload("er1000", scale=0.2)
    full = oracle.mine(g, 3, 1)
    a = oracle.mine(g, 3, 1, roots=(0, g.n // 2))
    b = oracle.mine(g, 3, 1, roots=(g.n // 2, g.n))
    tot = {}
    for part in (a, b):
        for l, adj, c in zip(part["labels"], part["adj"], part["count"]):
            key = (tuple(l), int(adj))
            tot[key] = tot.get(key, 0) + int(c)
    assert tot == {(tuple(l), int(adj)): int(c) for l, adj, c in zip(full["labels"], full["adj"], full["count"])}


def test_er1000_runs_quickly():
    g = gg.workload("er1000")
    o = oracle.mine(g, 3, 30)
    assert len(o["support"]) > 0
    assert np.all(o["support"] >= 30)
    # label sequences are nondecreasing in canonical order
    assert np.all(np.diff(o["labels"], axis=1) >= 0)


# --------------------------------------------------------------------- one-pattern matcher

@pytest.mark.parametrize("mode", ["edge", "vertex"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pattern_matcher_agrees_with_enumeration(mode, seed):
    """oracle.pattern_support (backtracking over label-preserving maps) and oracle.mine (ESU
    plus canonical codes) are independent; they must agree on every pattern."""
    g = gg.random_small(9, 0.4, 2, seed)
    for k in (1, 2, 3, 4, 5):
        o = oracle.mine(g, k, 1, mode)
        for lab, adj, s, c in zip(o["labels"], o["adj"], o["support"], o["count"]):
            assert oracle.pattern_support(g, lab, int(adj), mode) == (int(s), int(c))


def test_pattern_matcher_closed_forms():
    # path P_k inside P_9: sigma = 9 - 2*floor((k-1)/2), 9-k+1 embeddings
    for k in (2, 3, 4, 5):
        adj = sum(1 << (i * k + i + 1) for i in range(k - 1))
        assert oracle.pattern_support(gg.path(9), [0] * k, adj) == (9 - 2 * ((k - 1) // 2), 9 - k + 1)
    # triangle in K_5: sigma 5, C(5,3) embeddings; absent pattern gives (0, 0)
    assert oracle.pattern_support(gg.complete(5), [0, 0, 0], 2 + 4 + 32) == (5, 10)
    assert oracle.pattern_support(gg.path(6), [0, 0, 0], 2 + 4 + 32) == (0, 0)
    # star K_{1,3} centred at position 0 has 8 * 7 * 6 * 5 maps into K_8
    with pytest.raises(OverflowError):
        oracle.pattern_support(gg.complete(8), [0, 0, 0, 0], 2 + 4 + 8, max_maps=10)


# --------------------------------------------------------------------- network reference

def test_mlp_reference_gradient_matches_finite_differences():
    import oracle.mlp as mlp
    rng = np.random.default_rng(0)
    theta = rng.normal(0, 0.3, mlp.NPARAM)
    X = rng.normal(0, 1, (16, 32))
    Y = rng.normal(0, 1, 16)
    mu, sd = np.zeros(32), np.ones(32)
    p = mlp.unpack(theta)
    loss, g = mlp.loss_and_grad(p, X, Y, mu, sd)
    for idx in rng.choice(mlp.NPARAM, size=60, replace=False):
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[idx] += h
        tm[idx] -= h
        num = (mlp.loss_and_grad(mlp.unpack(tp), X, Y, mu, sd)[0] - mlp.loss_and_grad(mlp.unpack(tm), X, Y, mu, sd)[0]) / (2 * h)
        assert abs(num - g[idx]) <= 1e-6 + 1e-5 * abs(num), idx


def test_mlp_reference_closed_form():
    """With W1 = I on the first 32 units, W2 = I, w3 = e_0 and zero biases the network returns
    relu(x'_0); the loss against 0 is mean(relu(x_0)^2)."""
    import oracle.mlp as mlp
    parts = {"W1": np.eye(32, 64), "b1": np.zeros(64), "W2": np.eye(64), "b2": np.zeros(64),
             "w3": np.eye(64)[0], "b3": np.zeros(1)}
    X = np.zeros((4, 32))
    X[:, 0] = [-1.0, 0.5, 2.0, 3.0]
    y, _ = mlp.forward(parts, X, np.zeros(32), np.ones(32))
    assert np.allclose(y, [0.0, 0.5, 2.0, 3.0])
    loss, _ = mlp.loss_and_grad(parts, X, np.zeros(4), np.zeros(32), np.ones(32))
    assert np.isclose(loss, (0.25 + 4 + 9) / 4)


def test_bf16_rounding():
    import oracle.mlp as mlp
    # 1 + 2^-8 is halfway between bfloat16 neighbours 1 and 1 + 2^-7: ties to even gives 1
    assert mlp.bf16_round(np.float32(1 + 2 ** -8)) == 1.0
    assert mlp.bf16_round(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6
    assert mlp.bf16_round(np.float32(-2.0)) == -2.0


def test_adam_reference_first_step():
    """Adam's first bias-corrected step moves each weight by lr * sign(g) (up to eps)."""
    import oracle.mlp as mlp
    g = np.array([0.5, -2.0, 1e-3])
    th, m, v = mlp.adam_step(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, 0.01)
    assert np.allclose(th, -0.01 * np.sign(g), atol=1e-6)
