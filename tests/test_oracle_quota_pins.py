"""Pins for the oracle's quota-sampled mining (Section 5's fixed sampling thresholds taken
through the method's own steps), checked against things other than itself:

* with no quota it is exact mining, so it must equal the plain ESU oracle (a different
  enumeration: connected vertex sets grown from their smallest vertex, every edge subset) on
  random graphs for k = 3..7 and on the 1000-vertex Erdos-Renyi workload;
* a drawn embedding is an embedding, so every sampled support and count is a lower bound of the
  exact one, and every reported pattern is really frequent;
* the draw: a is coprime to c (Q distinct candidates) and is the first such value at or after
  1 + (h mod (c - 1)); each candidate is drawn with probability Q / c over the hash.
No GPU is used."""
import math

import numpy as np
import pytest

import graphgen as gg
import oracle

M64 = (1 << 64) - 1


def _same(a, b):
    return all(np.array_equal(a[x], b[x]) for x in ("labels", "adj", "support", "count"))


@pytest.mark.parametrize("mode", ["edge", "vertex"])
@pytest.mark.parametrize("seed", range(4))
def test_quota_oracle_without_quotas_is_exact(mode, seed):
    g = gg.random_small(9, 0.45, 2, seed)
    for k in range(3, 8 if seed == 0 else 7):
        assert _same(oracle.mine_quota(g, k, 1, mode), oracle.mine(g, k, 1, mode)), k


@pytest.mark.parametrize("k", [3, 4, 5])
def test_quota_oracle_without_quotas_is_exact_er1000(k):
    g = gg.workload("er1000")
    assert _same(oracle.mine_quota(g, k, 10), oracle.mine(g, k, 10))
    # quotas larger than every key group draw everything
    assert _same(oracle.mine_quota(g, k, 10, seed=5, join_quota=10 ** 4, match_quota=10 ** 9), oracle.mine(g, k, 10))


_EXACT = {}


def _hub_graph():
    return gg.chung_lu(600, 1200, 2.1, 2, cap=48, num_labels=3, label_law="zipf", zipf_s=1.2)


@pytest.mark.parametrize("mode", ["edge", "vertex"])
@pytest.mark.parametrize("k,x,m", [(3, 0, 20), (4, 2, 0), (4, 3, 40), (5, 3, 0), (5, 4, 60)])
def test_quota_results_are_lower_bounds(mode, k, x, m):
    # the 100k-vertex workload's shape at 1/200 scale for k <= 4; a sparse graph with hubs of
    # degree up to 50 for k = 5, where the exact oracle still takes seconds
    g = gg.workload("cl100k", scale=0.005, cap=30) if k <= 4 else _hub_graph()
    t = 6
    key = (g.content_hash(), k, mode)
    if key not in _EXACT:
        _EXACT[key] = oracle.mine(g, k, 1, mode)
    ex = _EXACT[key]
    idx = {(tuple(int(v) for v in l), int(a)): i for i, (l, a) in enumerate(zip(ex["labels"], ex["adj"]))}
    q = oracle.mine_quota(g, k, t, mode, seed=11, join_quota=x, match_quota=m)
    assert len(q["support"]) > 0
    assert np.all(q["support"] >= t)
    for l, a, s, c in zip(q["labels"], q["adj"], q["support"], q["count"]):
        i = idx[(tuple(int(v) for v in l), int(a))]
        assert s <= ex["support"][i] and c <= ex["count"][i]
        assert ex["support"][i] >= t
    assert int(q["count"].sum()) < int(ex["count"][ex["support"] >= t].sum())


def test_quota_draw_is_the_first_coprime_stride():
    rng = np.random.default_rng(4)
    for _ in range(3000):
        h = int(rng.integers(0, 2 ** 63)) * 2 + int(rng.integers(0, 2))
        c = int(rng.choice([2, 3, 6, 12, 30, 97, 210, 1024, 30030, 2 ** 20 + 7]))
        a, b = oracle.quota_draw(h, c)
        assert 1 <= a < c and 0 <= b < c and math.gcd(a, c) == 1
        x = 1 + h % (c - 1)
        while x != a:                 # every value skipped on the way shares a factor with c
            assert math.gcd(x, c) != 1
            x = 1 if x + 1 == c else x + 1


def test_quota_draw_takes_distinct_candidates_uniformly():
    c, Q, trials = 40, 8, 4000
    hits = np.zeros(c)
    rng = np.random.default_rng(5)
    for _ in range(trials):
        a, b = oracle.quota_draw(int(rng.integers(0, 2 ** 63)), c)
        drawn = {(a * j + b) % c for j in range(Q)}
        assert len(drawn) == Q
        hits[list(drawn)] += 1
    p = Q / c
    assert np.all(np.abs(hits - trials * p) <= 5 * math.sqrt(trials * p * (1 - p)))
