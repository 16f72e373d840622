"""The seeded input generators: CSR invariants, determinism, the recorded shape of the
benchmark graph, and the label laws.  CPU only."""
import numpy as np
import pytest

import graphgen as gg


def _check_csr(g):
    rp, col = g.row_ptr, g.col
    assert rp.dtype == np.int32 and col.dtype == np.int32 and g.labels.dtype == np.int32
    assert rp[0] == 0 and rp[-1] == col.size and np.all(np.diff(rp) >= 0)
    src = np.repeat(np.arange(g.n), np.diff(rp))
    assert np.all(src != col)                                    # no self-loops
    for v in range(0, g.n, max(1, g.n // 200)):                  # rows sorted, no duplicates
        row = col[rp[v]:rp[v + 1]]
        assert np.all(np.diff(row) > 0)
    fwd = set(zip(src.tolist(), col.tolist()))                   # symmetric
    assert all((w, u) in fwd for u, w in list(fwd)[:20000])
    assert g.labels.min() >= 0 and g.labels.max() < g.num_labels


@pytest.mark.parametrize("name,scale", [("er1000", 1.0), ("cl100k", 0.01), ("cl3700k", 0.0005), ("cl1100k", 0.002)])
def test_workloads_are_valid_csr(name, scale):
    _check_csr(gg.workload(name, scale=scale))


@pytest.mark.parametrize("g", [gg.complete(6), gg.path(7), gg.cycle(9), gg.star(5), gg.complete_bipartite(3, 4),
                               gg.spider(3, 2)])
def test_closed_forms_are_valid_csr(g):
    _check_csr(g)


def test_closed_form_edge_counts():
    assert gg.complete(6).m == 15
    assert gg.path(7).m == 6
    assert gg.cycle(9).m == 9
    assert gg.star(5).m == 5
    assert gg.complete_bipartite(3, 4).m == 12


def test_seeded_and_deterministic():
    a = gg.workload("cl100k", scale=0.01)
    b = gg.workload("cl100k", scale=0.01)
    c = gg.workload("cl100k", scale=0.01, seed=7)
    assert a.content_hash() == b.content_hash()
    assert a.content_hash() != c.content_hash()


def test_benchmark_graph_is_the_recorded_one():
    """The bench graph (100k vertices, 1.1M edges, beta 2.1, 29 Zipf(1.2) labels, seed 1,
    degree cap 300) is exactly the graph every recorded bench line was measured on."""
    g = gg.workload("cl100k", cap=300.0)
    assert (g.n, g.m) == (100000, 1100000)
    assert int(g.degrees().max()) == 358
    assert g.content_hash() == "fabe93f15ce93b12"


def test_chung_lu_has_m_edges_and_heavy_tail():
    g = gg.chung_lu(20000, 100000, 2.1, seed=3)
    assert g.m == 100000
    d = g.degrees()
    assert d.max() > 10 * d.mean()          # power-law hubs
    assert np.median(d) < d.mean()          # skewed to the right


def test_zipf_labels_follow_the_law():
    s, L, n = 1.2, 29, 400000
    lab = gg.zipf_labels(n, L, s, np.random.default_rng(5))
    freq = np.bincount(lab, minlength=L) / n
    expect = (np.arange(L) + 1.0) ** -s
    expect /= expect.sum()
    assert np.abs(freq - expect).max() < 0.01


def test_uniform_labels_are_uniform():
    lab = gg.uniform_labels(320000, 16, np.random.default_rng(2))
    freq = np.bincount(lab, minlength=16) / lab.size
    assert np.abs(freq - 1 / 16).max() < 0.005
