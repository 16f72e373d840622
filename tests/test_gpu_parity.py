"""GPU parity: the CUDA library against the CPU oracle, bit-exact (same patterns, same MNI
supports, same embedding counts), through the C ABI."""
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


def _same(got, exp, ctx=""):
    assert got["labels"].shape == exp["labels"].shape, f"{ctx}: {got['labels'].shape[0]} patterns vs oracle {exp['labels'].shape[0]}"
    for key in ("labels", "adj", "support", "count"):
        if not np.array_equal(got[key], exp[key]):
            bad = np.nonzero(np.any(np.atleast_2d(got[key] != exp[key]).reshape(len(got["support"]), -1), axis=1))[0][:5]
            raise AssertionError(f"{ctx}: {key} differs at rows {bad.tolist()}: "
                                 f"got {got[key][bad].tolist()} expected {exp[key][bad].tolist()}")


_ORACLE = {}


def oracle_at(g, k, t, mode="edge"):
    """Oracle result at threshold t.  The oracle computes every pattern's support without
    pruning, so one run at t=1 filtered by support >= t equals a run at t."""
    key = (g.content_hash(), k, mode)
    if key not in _ORACLE:
        _ORACLE[key] = oracle.mine(g, k, 1, mode)
    full = _ORACLE[key]
    keep = full["support"] >= t
    return {name: arr[keep] for name, arr in full.items()}


def check(fsm, g, k, t, mode="edge", options=None):
    G = fsm.Graph.from_graphgen(g, mode)
    for key, val in (options or {}).items():
        G.set_option(key, val)
    got = G.mine(k, t)
    G.close()
    exp = oracle_at(g, k, t, mode)
    _same(got, exp, f"k={k} t={t} mode={mode} n={g.n}")
    return got


@pytest.mark.parametrize("mode", ["edge", "vertex"])
@pytest.mark.parametrize("seed", range(6))
def test_tiny_random(fsm, mode, seed):
    g = gg.random_small(10, 0.35, 1 + seed % 3, seed)
    for k in range(1, 7):
        check(fsm, g, k, 1, mode)


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_closed_forms(fsm, mode):
    for k in range(1, 7):
        check(fsm, gg.complete(7), k, 1, mode)
        check(fsm, gg.path(12), k, 1, mode)
        check(fsm, gg.cycle(9), k, 1, mode)
        check(fsm, gg.star(7), k, 1, mode)
    check(fsm, gg.complete_bipartite(3, 5), 2, 1, mode)
    check(fsm, gg.spider(3, 2), 7, 1, mode)


def test_complete_graph_pattern_counts(fsm):
    # edge-induced K_7 at k = 6: all 112 connected 6-vertex graphs, each with sigma = 7
    got = check(fsm, gg.complete(7), 6, 1, "edge")
    assert len(got["support"]) == 112 and np.all(got["support"] == 7)


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_er1000_config(fsm, mode):
    """Erdos-Renyi n=1000, average degree 6, 4 uniform labels, threshold 30 (k <= 3), plus k=4."""
    g = gg.workload("er1000")
    for k in (1, 2, 3, 4):
        check(fsm, g, k, 30, mode)


@pytest.mark.parametrize("k", [5, 6, 7, 8])
def test_large_k_sparse(fsm, k):
    n = 40 if k <= 7 else 20
    g = gg.erdos_renyi(n, 2.5, seed=k, num_labels=2)
    for mode in ("edge", "vertex"):
        check(fsm, g, k, 1, mode)
        check(fsm, g, k, 3, mode)


@pytest.mark.parametrize("t", [2, 6, 20])
def test_chung_lu_scaled(fsm, t):
    """Shape of the 100k-vertex Chung-Lu workload (beta 2.1, 29 Zipf labels) at 1/200 scale."""
    g = gg.workload("cl100k", scale=0.005, cap=30)
    for k in (3, 4):
        check(fsm, g, k, t)


def test_chunking_and_batching_do_not_change_results(fsm):
    g = gg.workload("cl100k", scale=0.005, cap=30)
    ref = check(fsm, g, 4, 6)
    for opts in ({"chunk": 32}, {"chunk": 65536}, {"batch": 1024}, {"batch": 1024, "chunk": 64},
                 {"autotune": 1}, {"autotune": 1, "launch": 1}, {"launch": 1, "group": 1},
                 {"fused": 0}, {"fused": 0, "launch": 2},
                 {"fused_pool": 64}, {"fused_pool": 4096, "launch": 1}):
        G = fsm.Graph.from_graphgen(g)
        for key, val in opts.items():
            G.set_option(key, val)
        got = G.mine(4, 6)
        G.close()
        _same(got, ref, str(opts))


def test_deterministic_and_reusable_handle(fsm):
    g = gg.workload("er1000")
    G = fsm.Graph.from_graphgen(g)
    a = G.mine(4, 10)
    b = G.mine(4, 10)
    c = G.mine(3, 30)
    G.close()
    for key in a:
        assert np.array_equal(a[key], b[key])
    _same(c, oracle_at(g, 3, 30), "after reuse")


def test_vertex_renaming(fsm):
    g = gg.workload("cl100k", scale=0.01, cap=40)
    h = gg.relabel_vertices(g, np.random.default_rng(3).permutation(g.n))
    Gg, Gh = fsm.Graph.from_graphgen(g), fsm.Graph.from_graphgen(h)
    a, b = Gg.mine(4, 3), Gh.mine(4, 3)
    Gg.close()
    Gh.close()
    for key in a:
        assert np.array_equal(a[key], b[key])


def test_errors(fsm):
    g = gg.path(5)
    G = fsm.Graph.from_graphgen(g)
    with pytest.raises(fsm.FsmError) as e:
        G.mine(10, 1)
    assert e.value.code == fsm.FSM_EINVAL
    with pytest.raises(fsm.FsmError) as e:
        G.mine(3, 0)
    assert e.value.code == fsm.FSM_EINVAL
    with pytest.raises(fsm.FsmError) as e:
        G.mine(3, 1, sample_rate=0.0)
    assert e.value.code == fsm.FSM_EINVAL
    with pytest.raises(fsm.FsmError) as e:
        G.mine(3, 1, sample_rate=1.5)
    assert e.value.code == fsm.FSM_EINVAL
    with pytest.raises(fsm.FsmError):
        G.set_option("mode", 2)
    G.close()
    # asymmetric CSR
    with pytest.raises(fsm.FsmError) as e:
        fsm.fsm_load_graph(np.array([0, 1, 1], np.int32), np.array([1], np.int32), np.zeros(2, np.int32), 2, 1)
    assert e.value.code == fsm.FSM_EINVAL
    # unsorted row
    with pytest.raises(fsm.FsmError) as e:
        fsm.fsm_load_graph(np.array([0, 2, 3, 4], np.int32), np.array([2, 1, 0, 0], np.int32), np.zeros(3, np.int32), 3, 1)
    assert e.value.code == fsm.FSM_EINVAL


def test_stats(fsm):
    g = gg.workload("er1000")
    G = fsm.Graph.from_graphgen(g)
    r = G.mine(4, 30, stats=True)
    G.close()
    s = r["stats"]
    assert s["levels"] == 2 and s["kernel_launches"] > 0 and s["time_ns"] > 0
    # every returned embedding was accepted in the last level
    assert s["final_embeddings"] >= int(r["count"].sum())


@pytest.mark.parametrize("fused", [0, 1])
def test_fused_and_two_pass_last_level(fsm, fused):
    for g, k, t in [(gg.workload("er1000"), 3, 30), (gg.workload("er1000"), 4, 10),
                    (gg.erdos_renyi(40, 2.5, seed=7, num_labels=2), 6, 2)]:
        for mode in ("edge", "vertex"):
            check(fsm, g, k, t, mode, {"fused": fused})


@pytest.mark.parametrize("launch", [0, 1, 2])
def test_launch_modes_identical(fsm, launch):
    """Batched, persistent (one work-stealing launch per pass, CUDA-graph captured) and
    per-pattern launches give the oracle's result."""
    cases = [(gg.workload("er1000"), 4, 10), (gg.workload("er1000"), 5, 10),
             (gg.workload("cl100k", scale=0.005, cap=30), 4, 6),
             (gg.erdos_renyi(40, 2.5, seed=7, num_labels=2), 7, 2)]
    for g, k, t in cases:
        opts = {"launch": launch}
        check(fsm, g, k, t, "edge", opts)
        check(fsm, g, k, t, "edge", dict(opts, batch=1024, chunk=64))
        check(fsm, g, k, t, "vertex", opts)
        if launch == 1:
            check(fsm, g, k, t, "edge", dict(opts, group=1))
            check(fsm, g, k, t, "edge", dict(opts, group=0))


def test_autotune_picks_a_candidate_and_keeps_results(fsm):
    g = gg.workload("cl100k", scale=0.005, cap=30)
    G = fsm.Graph.from_graphgen(g)
    G.set_option("autotune", 1)
    a = G.mine(4, 6, stats=True)
    b = G.mine(4, 6, stats=True)
    G.close()
    assert a["stats"]["chunk_l2"] in (256, 1024, 4096, 16384)
    assert b["stats"]["chunk_l2"] == a["stats"]["chunk_l2"]
    _same(a, oracle_at(g, 4, 6), "autotuned")
    _same(b, oracle_at(g, 4, 6), "autotuned, second call")


def test_profile_option_counts_launches(fsm):
    g = gg.workload("er1000")
    G = fsm.Graph.from_graphgen(g)
    G.set_option("profile", 1)
    for launch in (0, 1, 2):
        G.set_option("launch", launch)
        r = G.mine(5, 10, stats=True)
        s = r["stats"]
        assert s["count_launches_l3"] >= 1 and s["count_ns_l3"] > 0 and s["count_bytes_l3"] > 0
        assert s["domain_launches_l1"] >= 1 and s["emit_launches_l1"] >= 1
    G.set_option("fused", 1)
    s = G.mine(5, 10, stats=True)["stats"]
    # the last level (3 -> 5) is then one fused pass
    assert s["fused_launches_l3"] >= 1 and s["fused_ns_l3"] > 0 and s["fused_bytes_l3"] > 0
    G.close()


@pytest.mark.parametrize("shape", [("cl3700k", 0.00012, 12), ("cl1100k", 0.0008, 12)])
def test_config_shaped_graphs_k5(fsm, shape):
    """Chung-Lu graphs shaped like the 3.7M-vertex workload (beta 2.3, 37 Zipf labels) and the
    1.1M-vertex one (beta 2.0, 16 uniform labels), scaled to about a thousand vertices, k = 5."""
    name, scale, cap = shape
    g = gg.workload(name, scale=scale, cap=cap)
    for t in (2, 4):
        check(fsm, g, 5, t, "edge", {"launch": 1})


def _hub_graph():
    """600 vertices, 1200 edges, degree cap 48 (beta 2.1, 3 Zipf labels): 13 vertices of degree
    >= 32, so five-vertex joins from stored triples meet the paths the full-size workloads take
    on hub key vertices -- neighbour matrices for the triangle test and shared-memory cross
    masks of single-unit chunks -- while the oracle still finishes in seconds."""
    return gg.chung_lu(600, 1200, 2.1, 2, cap=48, num_labels=3, label_law="zipf", zipf_s=1.2)


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_hub_graph_k5(fsm, mode):
    g = _hub_graph()
    assert int((g.degrees() >= 32).sum()) >= 10
    for t in (1, 40):
        for opts in ({"launch": 1}, {"launch": 0, "chunk": 32}, {"launch": 2}, {"launch": 1, "chunk": 4096}):
            check(fsm, g, 5, t, mode, opts)


@pytest.mark.parametrize("k", [3, 4])
def test_quick_pattern_table_overflow_and_retry(fsm, k):
    """A 64-slot first table overflows at once: every level grows it x4 and repeats its count
    pass until it fits, with the oracle's result."""
    g = gg.workload("cl100k", scale=0.005, cap=30)
    G = fsm.Graph.from_graphgen(g)
    G.set_option("qp_capacity", 64)
    got = G.mine(k, 6, stats=True)
    G.close()
    assert got["stats"]["qp_grows"] >= 2
    _same(got, oracle_at(g, k, 6), f"qp_capacity=64 k={k}")


@pytest.mark.parametrize("opts", [{"explore": 1}, {"quick_pattern": 1}])
@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_exploration_ablations_match_oracle(fsm, opts, mode):
    """Section 6's ablations -- single-vertex exploration (l -> l+1) and edge-list quick
    patterns -- compute the same exact result as the method itself, in every launch mode."""
    cases = [(gg.random_small(10, 0.35, 2, 3), range(2, 7), 1),
             (gg.workload("er1000"), (2, 3, 4, 5), 10),
             (gg.workload("cl100k", scale=0.005, cap=30), (3, 4), 6),
             (_hub_graph(), (4, 5), 40)]
    for g, ks, t in cases:
        for k in ks:
            check(fsm, g, k, t, mode, dict(opts, launch=1))
    g = gg.workload("er1000")
    for launch in (0, 2):
        check(fsm, g, 4, 10, mode, dict(opts, launch=launch))


def test_ablation_counters(fsm):
    """Edge-list quick patterns canonicalise more distinct keys than index-based ones for the
    same output; single-vertex exploration runs one level per added vertex."""
    g = gg.workload("cl100k", scale=0.005, cap=30)
    G = fsm.Graph.from_graphgen(g)
    ref = G.mine(4, 6, stats=True)
    G.set_option("quick_pattern", 1)
    el = G.mine(4, 6, stats=True)
    G.set_option("quick_pattern", 0)
    G.set_option("explore", 1)
    sv = G.mine(4, 6, stats=True)
    with pytest.raises(fsm.FsmError) as e:
        G.mine(4, 6, sample_rate=0.5)
    assert e.value.code == fsm.FSM_EUNSUPPORTED
    G.close()
    for r in (el, sv):
        for key in ("labels", "adj", "support", "count"):
            assert np.array_equal(r[key], ref[key])
    assert el["stats"]["quick_patterns"] > ref["stats"]["quick_patterns"]
    assert ref["stats"]["levels"] == 2 and sv["stats"]["levels"] == 3


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_one_pass_last_level(fsm, mode):
    """Option fused = 1: the last level counted and its domains filled in one enumeration, with
    quick patterns canonicalised on first sight in the kernel -- the oracle's result, also when
    a small bitmap pool forces the count-and-domain fallback."""
    for g, k, t in [(_hub_graph(), 5, 40), (gg.workload("er1000"), 5, 10), (gg.workload("er1000"), 3, 30),
                    (gg.erdos_renyi(40, 2.5, seed=7, num_labels=2), 7, 2), (gg.workload("cl100k", scale=0.005, cap=30), 4, 6)]:
        for launch in (0, 1, 2):
            check(fsm, g, k, t, mode, {"fused": 1, "launch": launch})
    G = fsm.Graph.from_graphgen(_hub_graph(), mode)
    G.set_option("fused", 1)
    G.set_option("fused_pool", 64)
    got = G.mine(5, 40, stats=True)
    G.close()
    assert got["stats"]["fused_fallbacks"] >= 1
    _same(got, oracle_at(_hub_graph(), 5, 40, mode), "fused fallback")


def test_debug_option_keeps_results(fsm):
    """Option debug = 1 bounds-checks every decoded list index in the kernels (flag and skip,
    never trap); on valid input nothing trips and the result is the oracle's."""
    for g, k, t in [(gg.workload("er1000"), 4, 10), (_hub_graph(), 5, 40)]:
        for opts in ({"debug": 1, "launch": 1}, {"debug": 1, "explore": 1}, {"debug": 1, "fused": 1}):
            check(fsm, g, k, t, "edge", opts)


def test_time_limit_returns_etimeout_and_the_handle_recovers(fsm):
    """A call past option time_limit_ms stops taking work at the next chunk and returns
    FSM_ETIMEOUT; the same handle then mines normally."""
    g = gg.workload("cl100k", cap=100)
    G = fsm.Graph.from_graphgen(g)
    G.set_option("launch", 1)
    G.set_option("time_limit_ms", 20)
    with pytest.raises(fsm.FsmError) as e:
        G.mine(5, 300)
    assert e.value.code == fsm.FSM_ETIMEOUT
    G.set_option("time_limit_ms", 0)
    after = G.mine(4, 300)
    G.close()
    H = fsm.Graph.from_graphgen(g)
    H.set_option("launch", 1)
    fresh = H.mine(4, 300)
    H.close()
    for key in ("labels", "adj", "support", "count"):
        assert np.array_equal(after[key], fresh[key])


def test_injected_allocation_failure_returns_enomem(fsm):
    g = gg.workload("er1000")
    G = fsm.Graph.from_graphgen(g)
    for n in (1, 5, 20, 40):
        G.set_option("fail_alloc_after", n)
        with pytest.raises(fsm.FsmError) as e:
            G.mine(4, 10)
        assert e.value.code == fsm.FSM_ENOMEM, n
    G.set_option("fail_alloc_after", 0)
    got = G.mine(4, 10)
    G.close()
    _same(got, oracle_at(g, 4, 10), "after injected allocation failures")


def _degenerate_graphs():
    return [
        ("one vertex", gg.from_edges(1, [], np.array([0], np.int32), 1), (1, 2, 3, 5), 1),
        ("isolated vertices", gg.from_edges(6, [], np.array([0, 1, 0, 1, 0, 1], np.int32), 2), (1, 2, 3, 4), 1),
        ("one edge", gg.from_edges(2, [(0, 1)], np.array([0, 1], np.int32), 2), (1, 2, 3, 4), 1),
        ("k above n", gg.path(5), (6, 7, 8, 9), 1),
        ("nothing frequent", gg.workload("er1000"), (2, 3, 4, 5), 10 ** 6),
    ]


@pytest.mark.parametrize("mode", ["edge", "vertex"])
def test_degenerate_inputs(fsm, mode):
    """Graphs without edges, a single edge, k above the vertex count and thresholds no pattern
    reaches: every exploration form, last-level form, launch mode and sampling mode returns the
    oracle's (mostly empty) answer."""
    for name, g, ks, t in _degenerate_graphs():
        for k in ks:
            for opts in ({}, {"launch": 0}, {"launch": 2}, {"fused": 1}, {"explore": 1}, {"quick_pattern": 1}):
                if k > 7 and ("explore" in opts or "quick_pattern" in opts):
                    continue
                check(fsm, g, k, t, mode, opts)
            if k >= 3:
                G = fsm.Graph.from_graphgen(g, mode)
                G.set_option("join_quota", 2)
                got = G.mine(k, t)
                G.set_option("join_quota", 0)      # rate sampling runs without quotas, k <= 8
                sampled = G.mine(k, t, sample_rate=0.5) if k <= 8 else {"support": []}
                G.close()
                exp = oracle.mine_quota(g, k, t, mode, seed=0, join_quota=2)
                for key in ("labels", "adj", "support", "count"):
                    assert np.array_equal(got[key], exp[key]), (name, k, key)
                assert len(sampled["support"]) <= max(1, len(oracle_at(g, k, 1, mode)["support"]))
