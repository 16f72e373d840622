"""Section 5's sampling with fixed thresholds on the GPU (options join_quota = ST x: x^2 candidate
pieces per key group and, joining edges, x edges per key vertex; match_quota = M.ST: candidate
pieces per vertex when size-3 subgraphs are matched), bit-exact against the oracle's
restatement of the same draws through the method's steps (oracle.mine_quota): same patterns,
same sampled supports and counts, in every launch mode and both induction modes."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fsm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_07690_gb300 import build, fsm as f
    build.build()
    f.load()
    return f


def _run(fsm, g, k, t, mode, seed, x, m, launch=1):
    G = fsm.Graph.from_graphgen(g, mode)
    G.set_option("seed", seed)
    G.set_option("join_quota", x)
    G.set_option("match_quota", m)
    G.set_option("launch", launch)
    r = G.mine(k, t)
    G.close()
    return r


def _check(fsm, g, k, t, mode, seed, x, m, launch=1):
    got = _run(fsm, g, k, t, mode, seed, x, m, launch)
    exp = oracle.mine_quota(g, k, t, mode, seed=seed, join_quota=x, match_quota=m)
    ctx = f"k={k} t={t} mode={mode} seed={seed} ST={x} M.ST={m} launch={launch}"
    assert got["labels"].shape == exp["labels"].shape, f"{ctx}: {len(got['support'])} vs {len(exp['support'])} patterns"
    for key in ("labels", "adj", "support", "count"):
        assert np.array_equal(got[key], exp[key]), f"{ctx}: {key} differs"
    assert np.all(got["exact"] == 0) or (x == 0 and m == 0)
    return got


def _hub_graph():
    return gg.chung_lu(600, 1200, 2.1, 2, cap=48, num_labels=3, label_law="zipf", zipf_s=1.2)


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_join_quota_matches_oracle(fsm, mode):
    cases = [(gg.workload("er1000"), (3, 4, 5), 10),
             (gg.workload("cl100k", scale=0.005, cap=30), (3, 4, 5), 6),
             (_hub_graph(), (4, 5), 20),
             (gg.random_small(12, 0.4, 2, 5), (4, 5, 6), 1)]
    for g, ks, t in cases:
        for k in ks:
            for x in (2, 3, 6):
                _check(fsm, g, k, t, mode, seed=7, x=x, m=0)


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_match_quota_matches_oracle(fsm, mode):
    g = gg.workload("cl100k", scale=0.005, cap=30)
    for k, x, m in ((3, 0, 15), (4, 3, 40), (5, 4, 25)):
        _check(fsm, g, k, 6, mode, seed=3, x=x, m=m)


@pytest.mark.parametrize("launch", [0, 2])
def test_quota_launch_modes(fsm, launch):
    g = gg.workload("cl100k", scale=0.005, cap=30)
    _check(fsm, g, 5, 6, "edge", seed=1, x=3, m=0, launch=launch)


def test_quota_draws_follow_the_seed(fsm):
    g = gg.workload("cl100k", scale=0.005, cap=30)
    a = _run(fsm, g, 4, 6, "edge", 1, 2, 0)
    b = _run(fsm, g, 4, 6, "edge", 2, 2, 0)
    assert not (np.array_equal(a["support"], b["support"]) and np.array_equal(a["count"], b["count"]))
    full = _run(fsm, g, 4, 6, "edge", 1, 0, 0)
    assert int(a["count"].sum()) < int(full["count"].sum())
