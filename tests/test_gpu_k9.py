"""Mining 9-vertex patterns on the GPU (Section 6, Table 3: 9-FSM with two-vertex exploration,
exactly and with ST x join quotas), bit-exact against the oracle: sparse labeled graphs whose
connected 9-vertex subgraphs the oracle can enumerate, one with a single label (every vertex
order label-preserving: the canonicaliser's cell search), every launch mode, bounds-checked
mode, both induction modes; and the k = 9 restrictions of the C ABI."""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu

K = 9


@pytest.fixture(scope="module")
def fsm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_07690_gb300 import build, fsm as f
    build.build()
    f.load()
    return f


_ORACLE = {}


def _oracle(g, mode, t):
    key = (g.content_hash(), mode)
    if key not in _ORACLE:
        _ORACLE[key] = oracle.mine(g, K, 1, mode)
    full = _ORACLE[key]
    keep = full["support"] >= t
    return {name: arr[keep] for name, arr in full.items()}


def _same(got, exp, ctx):
    assert got["labels"].shape == exp["labels"].shape, f"{ctx}: {len(got['support'])} vs {len(exp['support'])} patterns"
    for key in ("labels", "adj", "support", "count"):
        assert np.array_equal(got[key], exp[key]), f"{ctx}: {key} differs"


GRAPHS = [("tree+3, 3 labels", lambda: gg.tree_plus(13, 3, 3, 0)),
          ("tree+4, 2 labels", lambda: gg.tree_plus(13, 4, 2, 1)),
          ("tree+3, 1 label", lambda: gg.tree_plus(12, 3, 1, 2)),
          ("cycle 11", lambda: gg.cycle(11)),
          ("path 14", lambda: gg.path(14))]


@pytest.mark.parametrize("mode", ["edge", "vertex"])
@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_k9_matches_oracle(fsm, mode, gi):
    name, make = GRAPHS[gi]
    g = make()
    exp1 = _oracle(g, mode, 1)
    assert len(exp1["support"]) > 0
    for opts in ({}, {"launch": 0}, {"launch": 2}, {"debug": 1}):
        for t in (1, 2, 3):
            G = fsm.Graph.from_graphgen(g, mode)
            for key, val in opts.items():
                G.set_option(key, val)
            got = G.mine(K, t)
            G.close()
            assert got["adj"].dtype == object
            _same(got, _oracle(g, mode, t), f"{name} mode={mode} t={t} {opts}")


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_k9_join_quota_matches_oracle(fsm, mode):
    g = gg.tree_plus(14, 4, 2, 3)
    for x, m in ((2, 0), (3, 0), (2, 4)):
        G = fsm.Graph.from_graphgen(g, mode)
        G.set_option("seed", 7)
        G.set_option("join_quota", x)
        G.set_option("match_quota", m)
        got = G.mine(K, 1)
        G.close()
        exp = oracle.mine_quota(g, K, 1, mode, seed=7, join_quota=x, match_quota=m)
        _same(got, exp, f"mode={mode} ST={x} M.ST={m}")
        assert np.all(got["exact"] == 0)


def test_k9_restrictions(fsm):
    g = gg.tree_plus(12, 3, 2, 4)
    G = fsm.Graph.from_graphgen(g, "edge")
    try:
        for key in ("explore", "quick_pattern"):
            G.set_option(key, 1)
            with pytest.raises(fsm.FsmError) as e:
                G.mine(K, 1)
            assert e.value.code == fsm.FSM_EUNSUPPORTED
            G.set_option(key, 0)
        with pytest.raises(fsm.FsmError) as e:
            G.mine(K, 1, sample_rate=0.5)
        assert e.value.code == fsm.FSM_EUNSUPPORTED
        with pytest.raises(fsm.FsmError) as e:
            G.mine(K + 1, 1)
        assert e.value.code == fsm.FSM_EINVAL
        # the bit (i*k + j) word does not hold 9 vertices; the pair words do
        import ctypes
        r = ctypes.c_void_p()
        fsm._check(fsm.load().fsm_mine(G.handle, K, 1, 1.0, ctypes.byref(r)))
        try:
            assert fsm.fsm_result_count(r.value) > 0
            with pytest.raises(fsm.FsmError) as e:
                fsm.fsm_result_get(r.value, 0, K)
            assert e.value.code == fsm.FSM_EUNSUPPORTED
            pairs = fsm.fsm_result_pairs(r.value)
            assert np.all(pairs < (1 << 36)) and np.all(pairs > 0)
        finally:
            fsm.fsm_free_result(r.value)
    finally:
        G.close()
