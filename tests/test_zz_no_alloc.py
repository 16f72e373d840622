"""fsm_edge_supports_noalloc against fsm_mine(k=2), through the C ABI.

The entry point serves callers that cannot allocate device memory (code inside an allocator's
own callback, or a process whose device memory another framework's pool has reserved): it
keeps its scratch in one static device array.  Its supports and counts of every labeled edge
pattern must equal those that fsm_mine returns for k = 2 at threshold 1, on two calls in a row
(the array keeps the previous call's contents, so the second call checks that the entry point
clears what it reuses).  The file name makes pytest collect it last.
"""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_07690_gb300 import build, fsm
    build.build()
    fsm.load()
    return fsm, torch


def _noalloc(fsm, torch, g):
    dev = torch.device("cuda")
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    lab = torch.from_numpy(g.labels).to(dev)
    nl = g.num_labels
    sup = torch.full((nl * nl,), -1, dtype=torch.int64, device=dev)
    cnt = torch.full((nl * nl,), -1, dtype=torch.int64, device=dev)
    fsm.fsm_edge_supports_noalloc(rp.data_ptr(), col.data_ptr(), lab.data_ptr(), g.n, nl,
                                  sup.data_ptr(), cnt.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return sup.cpu().numpy(), cnt.cpu().numpy()


def _expected(fsm, g):
    G = fsm.Graph.from_graphgen(g)
    r = G.mine(2, 1)
    G.close()
    nl = g.num_labels
    sup = np.zeros(nl * nl, np.int64)
    cnt = np.zeros(nl * nl, np.int64)
    for lab, s, c in zip(r["labels"], r["support"], r["count"]):
        sup[lab[0] * nl + lab[1]] = s
        cnt[lab[0] * nl + lab[1]] = c
    return sup, cnt


GRAPHS = {
    "er1000": lambda: gg.workload("er1000"),
    "cl100k_scaled": lambda: gg.workload("cl100k", scale=0.05, cap=100),
    "cl100k_cap300": lambda: gg.workload("cl100k", cap=300),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_noalloc_matches_fsm_mine_on_two_calls(env, name):
    fsm, torch = env
    g = GRAPHS[name]()
    exp_sup, exp_cnt = _expected(fsm, g)
    for call in range(2):
        sup, cnt = _noalloc(fsm, torch, g)
        assert np.array_equal(sup, exp_sup), f"call {call}: supports differ"
        assert np.array_equal(cnt, exp_cnt), f"call {call}: counts differ"


def test_noalloc_rejects_graphs_beyond_its_scratch(env):
    fsm, _ = env
    # rejected on the host from the sizes alone, before any device work
    with pytest.raises(fsm.FsmError) as e:
        fsm.fsm_edge_supports_noalloc(1, 1, 1, 2 ** 30, 64, 1, 1, 0)
    assert e.value.code == fsm.FSM_EUNSUPPORTED
    assert "static array" in str(e.value)


# Malformed row_ptr arrays (path 0-1-2-3, nnz = 6) that the device validation must reject
# before reading outside col: a row that ends before it starts, a row that ends past nnz, a
# row that starts below zero, and a first row that does not start at 0.
BAD_ROW_PTRS = {
    "decreasing": [0, 4, 3, 5, 6],
    "past_nnz": [0, 1, 9, 5, 6],
    "negative": [0, -1, 3, 5, 6],
    "first_not_zero": [1, 1, 3, 5, 6],
}


@pytest.mark.parametrize("name", list(BAD_ROW_PTRS))
def test_noalloc_rejects_malformed_row_ptr(env, name):
    fsm, torch = env
    dev = torch.device("cuda")
    rp = torch.tensor(BAD_ROW_PTRS[name], dtype=torch.int32, device=dev)
    col = torch.tensor([1, 0, 2, 1, 3, 2], dtype=torch.int32, device=dev)
    lab = torch.zeros(4, dtype=torch.int32, device=dev)
    sup = torch.zeros(1, dtype=torch.int64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    with pytest.raises(fsm.FsmError) as e:
        fsm.fsm_edge_supports_noalloc(rp.data_ptr(), col.data_ptr(), lab.data_ptr(), 4, 1, sup.data_ptr(),
                                      cnt.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert e.value.code == fsm.FSM_EINVAL
    # the context is still usable: a valid call on the same path graph succeeds afterwards
    rp_ok = torch.tensor([0, 1, 3, 5, 6], dtype=torch.int32, device=dev)
    fsm.fsm_edge_supports_noalloc(rp_ok.data_ptr(), col.data_ptr(), lab.data_ptr(), 4, 1, sup.data_ptr(),
                                  cnt.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert int(sup.item()) == 4 and int(cnt.item()) == 3
