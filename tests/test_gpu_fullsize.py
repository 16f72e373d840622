"""Parity at the benchmark's full size: the 100k-vertex Chung-Lu graph (1.1M edges, beta 2.1,
29 Zipf labels, degree cap 300), k = 4, t = 300, in the launch configuration bench.py times
(persistent launch, autotuned chunks).  The oracle cannot enumerate all 1.6e10 embeddings, so
sampled output patterns are recomputed one by one by the oracle's pattern matcher (support and
embedding count, exactly), patterns one edit away from the output are checked to be really
infrequent, and properties that hold at any size are checked on the whole output."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

K, T = 4, 300
MAX_MAPS = 3_000_000


@pytest.fixture(scope="module")
def mined():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_07690_gb300 import build, fsm
    build.build()
    fsm.load()
    g = gg.workload("cl100k", cap=300)
    G = fsm.Graph.from_graphgen(g)
    G.set_option("launch", 1)
    G.set_option("autotune", 1)
    r = G.mine(K, T, stats=True)
    r3 = G.mine(3, T)
    G.set_option("launch", 0)
    r0 = G.mine(K, T)
    G.close()
    return g, r, r3, r0


def _edges(adj, k):
    return [(i, j) for i in range(k) for j in range(i + 1, k) if int(adj) >> (i * k + j) & 1]


def test_sampled_patterns_match_the_matcher(mined):
    g, r, _, _ = mined
    n = len(r["support"])
    assert n > 1000
    rng = np.random.default_rng(0)
    small = np.argsort(r["count"], kind="stable")[:4]
    light = np.nonzero(r["count"] <= MAX_MAPS // 24)[0]
    picks = list(small) + list(rng.choice(light, size=min(8, len(light)), replace=False))
    for q in picks:
        lab = [int(x) for x in r["labels"][q]]
        s, c = oracle.pattern_support(g, lab, int(r["adj"][q]), "edge", max_maps=MAX_MAPS)
        assert (s, c) == (int(r["support"][q]), int(r["count"][q])), (lab, _edges(r["adj"][q], K))


def test_neighbouring_patterns_absent_are_infrequent(mined):
    """Relabel one vertex of an output pattern: if the result is not in the output, the matcher
    must find its support below t."""
    g, r, _, _ = mined
    have = {(tuple(int(x) for x in l), int(a)) for l, a in zip(r["labels"], r["adj"])}
    rng = np.random.default_rng(1)
    checked = 0
    for q in rng.permutation(len(r["support"]))[:400]:
        lab = [int(x) for x in r["labels"][q]]
        pos = int(rng.integers(K))
        lab[pos] = int(rng.integers(g.num_labels))
        # canonical code of the edited pattern: mine the pattern graph itself (vertex-induced)
        pg = gg.from_edges(K, _edges(r["adj"][q], K), np.array(lab, np.int32), g.num_labels)
        o = oracle.mine(pg, K, 1, "vertex")
        key = (tuple(int(x) for x in o["labels"][0]), int(o["adj"][0]))
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
    g, r, r3, r0 = mined
    # identical across launch modes
    for key in ("labels", "adj", "support", "count"):
        assert np.array_equal(r[key], r0[key])
    # supports reach t, labels nondecreasing, rows sorted by (labels, adjacency sequence)
    assert np.all(r["support"] >= T)
    assert np.all(np.diff(r["labels"], axis=1) >= 0)
    pairs = [(i, j) for i in range(K) for j in range(i + 1, K)]
    keys = [tuple(int(x) for x in l) + tuple(int(a) >> (i * K + j) & 1 for i, j in pairs)
            for l, a in zip(r["labels"], r["adj"])]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    # MNI is anti-monotone: every connected 3-vertex sub-pattern is in the k = 3 output with
    # a support at least as large
    sup3 = {(tuple(int(x) for x in l), int(a)): int(s) for l, a, s in zip(r3["labels"], r3["adj"], r3["support"])}
    rng = np.random.default_rng(2)
    for q in rng.permutation(len(r["support"]))[:300]:
        lab = [int(x) for x in r["labels"][q]]
        edges = _edges(r["adj"][q], K)
        for drop in range(K):
            keep = [v for v in range(K) if v != drop]
            sub = [(keep.index(a), keep.index(b)) for a, b in edges if drop not in (a, b)]
            if len(sub) < 2:
                continue
            pg = gg.from_edges(3, sub, np.array([lab[v] for v in keep], np.int32), g.num_labels)
            o = oracle.mine(pg, 3, 1, "vertex")
            key = (tuple(int(x) for x in o["labels"][0]), int(o["adj"][0]))
            assert key in sup3 and sup3[key] >= int(r["support"][q])
