"""Parity at full size, in the launch configuration bench.py times (persistent launch,
autotuned chunks, one-pass last level on the benchmark workload), on two workloads:

* the 3.7M-vertex Chung-Lu graph (16.5M edges, beta 2.3, 37 Zipf(1.0) labels, degree cap 20),
  k = 5, t = 20000 -- the benchmark workload;
* the 100k-vertex Chung-Lu graph (1.1M edges, beta 2.1, 29 Zipf(1.2) labels, degree cap 300),
  k = 4, t = 300.

The oracle cannot enumerate 1e10 embeddings, so sampled output patterns (the smallest counts
and a random draw of light ones) are recomputed one by one by the oracle's pattern matcher
(support and embedding count, exactly), patterns one label edit away from the output are
checked to be really infrequent, and properties that hold at any size are checked on the whole
output: identical results from one launch per frontier pattern with the other last-level form
(two passes against one), sorted unique rows, supports reaching t, and anti-monotone supports
against the k = 3 output."""
import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

MAX_MAPS = 3_000_000
WORKLOADS = {
    "cl3700k_cap20_k5": dict(name="cl3700k", cap=20, k=5, t=20000, fused=1),
    "cl100k_cap300_k4": dict(name="cl100k", cap=300, k=4, t=300, fused=0),
}


@pytest.fixture(scope="module", params=list(WORKLOADS))
def mined(request):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_07690_gb300 import build, fsm
    build.build()
    fsm.load()
    w = WORKLOADS[request.param]
    g = gg.workload(w["name"], cap=w["cap"])
    G = fsm.Graph.from_graphgen(g)
    G.set_option("launch", 1)
    G.set_option("autotune", 1)
    G.set_option("fused", w["fused"])
    r = G.mine(w["k"], w["t"], stats=True)
    r3 = G.mine(3, w["t"])
    # the other launch mode and the other last-level form must agree
    G.set_option("launch", 2)
    G.set_option("fused", 1 - w["fused"])
    r2 = G.mine(w["k"], w["t"])
    G.close()
    return g, w["k"], w["t"], r, r3, r2


def _edges(adj, k):
    return [(i, j) for i in range(k) for j in range(i + 1, k) if int(adj) >> (i * k + j) & 1]


def _canonical(lab, edges, num_labels):
    """Canonical (labels, adj) of a small labeled graph: the oracle mining the graph itself
    (vertex-induced, k = its size)."""
    k = len(lab)
    pg = gg.from_edges(k, edges, np.array(lab, np.int32), num_labels)
    o = oracle.mine(pg, k, 1, "vertex")
    return tuple(int(x) for x in o["labels"][0]), int(o["adj"][0])


def test_sampled_patterns_match_the_matcher(mined):
    g, K, T, r, _, _ = mined
    n = len(r["support"])
    assert n > 1000
    rng = np.random.default_rng(0)
    small = np.argsort(r["count"], kind="stable")[:6]
    light = np.nonzero(r["count"] <= MAX_MAPS // 4)[0]
    picks = list(small) + list(rng.permutation(light))
    checked = 0
    for q in picks:
        lab = [int(x) for x in r["labels"][q]]
        try:
            s, c = oracle.pattern_support(g, lab, int(r["adj"][q]), "edge", max_maps=MAX_MAPS)
        except OverflowError:   # more label-preserving maps than the budget (automorphisms)
            continue
        assert (s, c) == (int(r["support"][q]), int(r["count"][q])), (lab, _edges(r["adj"][q], K))
        checked += 1
        if checked >= 14:
            break
    assert checked >= 12


def test_neighbouring_patterns_absent_are_infrequent(mined):
    """Relabel one vertex of an output pattern: if the result is not in the output, the matcher
    must find its support below t."""
    g, K, T, r, _, _ = mined
    have = {(tuple(int(x) for x in l), int(a)) for l, a in zip(r["labels"], r["adj"])}
    rng = np.random.default_rng(1)
    checked = 0
    for q in rng.permutation(len(r["support"]))[:400]:
        lab = [int(x) for x in r["labels"][q]]
        pos = int(rng.integers(K))
        lab[pos] = int(rng.integers(g.num_labels))
        key = _canonical(lab, _edges(r["adj"][q], K), g.num_labels)
        if key in have:
            continue
        try:
            s, _ = oracle.pattern_support(g, list(key[0]), key[1], "edge", max_maps=MAX_MAPS)
        except OverflowError:
            continue
        assert s < T, key
        checked += 1
        if checked >= 6:
            break
    assert checked >= 3


def test_properties_of_the_whole_output(mined):
    g, K, T, r, r3, r2 = mined
    # identical with one launch per frontier pattern and the other last-level form
    for key in ("labels", "adj", "support", "count"):
        assert np.array_equal(r[key], r2[key])
    # supports reach t, labels nondecreasing, rows sorted by (labels, adjacency sequence)
    assert np.all(r["support"] >= T)
    assert np.all(np.diff(r["labels"], axis=1) >= 0)
    pairs = [(i, j) for i in range(K) for j in range(i + 1, K)]
    keys = [tuple(int(x) for x in l) + tuple(int(a) >> (i * K + j) & 1 for i, j in pairs)
            for l, a in zip(r["labels"], r["adj"])]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    # MNI is anti-monotone: every connected 3-vertex sub-pattern is in the k = 3 output with a
    # support at least as large
    sup3 = {(tuple(int(x) for x in l), int(a)): int(s) for l, a, s in zip(r3["labels"], r3["adj"], r3["support"])}
    rng = np.random.default_rng(2)
    for q in rng.permutation(len(r["support"]))[:200]:
        lab = [int(x) for x in r["labels"][q]]
        edges = _edges(r["adj"][q], K)
        for keep in itertools.combinations(range(K), 3):
            sub = [(keep.index(a), keep.index(b)) for a, b in edges if a in keep and b in keep]
            if len(sub) < 2:
                continue
            key = _canonical([lab[v] for v in keep], sub, g.num_labels)
            assert key in sup3 and sup3[key] >= int(r["support"][q])
