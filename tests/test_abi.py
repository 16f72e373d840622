"""The C ABI without a GPU: the library loads, exports every declared entry point, rejects bad
arguments before touching a device, and its host build of the dissection rule matches the
paper's worked example and is total."""
import itertools
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fsm():
    from paper_2101_07690_gb300 import build, fsm as f
    build.build()
    f.load()
    return f


def test_exports_every_declared_symbol(fsm):
    header = open(os.path.join(ROOT, "include", "fsm.h")).read()
    declared = set(re.findall(r"^\s*(?:int|int64_t|void|const char \*)\s*\*?\s*(fsm_\w+)\s*\(", header, re.M))
    assert declared, "no declarations parsed"
    lib = fsm.load()
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(fsm.EXPORTS)


def test_bad_arguments_rejected_without_device(fsm):
    with pytest.raises(fsm.FsmError) as e:
        fsm.fsm_load_graph(np.array([0, 0], np.int32), np.zeros(0, np.int32), np.zeros(1, np.int32), 1, 0)
    assert e.value.code == fsm.FSM_EINVAL
    with pytest.raises(fsm.FsmError) as e:
        fsm.fsm_load_graph(np.array([1, 0], np.int32), np.zeros(1, np.int32), np.zeros(1, np.int32), 1, 1)
    assert e.value.code == fsm.FSM_EINVAL
    assert fsm.load().fsm_mine(None, 3, 1, 1.0, None) == fsm.FSM_EINVAL


def _read_cases():
    path = os.path.join(ROOT, "tests", "golden", "dissect_example.txt")
    cases = []
    for line in open(path):
        if line.startswith("case"):
            parts = [p.strip() for p in line[4:].split("|")]
            verts = [int(x) for x in parts[0].split()]
            edges = [tuple(int(y) for y in e.split("-")) for e in parts[1].split()]
            l_exp = [int(x) for x in parts[2].split()]
            cases.append((verts, edges, l_exp, int(parts[3])))
    return cases


@pytest.mark.parametrize("case", _read_cases())
def test_dissect_paper_example(fsm, case):
    verts, edges, l_exp, join_exp = case
    idx = {v: i for i, v in enumerate(verts)}
    rows = [0] * len(verts)
    for a, b in edges:
        rows[idx[a]] |= 1 << idx[b]
        rows[idx[b]] |= 1 << idx[a]
    lm, jn, fb = fsm.fsm_debug_dissect(verts, rows)
    assert sorted(v for v in verts if lm >> idx[v] & 1) == l_exp
    assert verts[jn] == join_exp
    assert fb == 0


def _connected(k, rows):
    seen, front = 1, 1
    while front:
        nx = 0
        for h in range(k):
            if front >> h & 1:
                nx |= rows[h]
        nx &= ~seen
        seen |= nx
        front = nx
    return seen == (1 << k) - 1


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_dissect_total_and_valid(fsm, k):
    """Every connected graph on k vertex ids has a dissection: a connected 3-vertex part l and
    a connected remainder sharing exactly the join vertex (Theorem 1)."""
    pairs = [(i, j) for i in range(k) for j in range(i + 1, k)]
    ids = list(range(k))
    fallbacks = 0
    for mask in range(1 << len(pairs)):
        rows = [0] * k
        for q, (a, b) in enumerate(pairs):
            if mask >> q & 1:
                rows[a] |= 1 << b
                rows[b] |= 1 << a
        if not _connected(k, rows):
            continue
        lm, jn, fb = fsm.fsm_debug_dissect(ids, rows)
        fallbacks += fb
        assert bin(lm).count("1") == 3 and lm >> jn & 1
        sub = lambda m: [rows[h] & m if m >> h & 1 else 0 for h in range(k)]
        # l connected
        lrows = sub(lm)
        lv = [h for h in range(k) if lm >> h & 1]
        assert sum(1 for a, b in itertools.combinations(lv, 2) if lrows[a] >> b & 1) >= 2
        # remainder plus join connected
        rm = (((1 << k) - 1) & ~lm) | (1 << jn)
        rrows = sub(rm)
        rv = [h for h in range(k) if rm >> h & 1]
        seen, front = 1 << rv[0], 1 << rv[0]
        while front:
            nx = 0
            for h in range(k):
                if front >> h & 1:
                    nx |= rrows[h]
            nx &= ~seen
            seen |= nx
            front = nx
        assert seen == rm
    print(f"k={k}: fallback rule used {fallbacks} times")


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_dissect_agrees_with_oracle(fsm, k):
    """The library's dissection rule and the oracle's (both written from Algorithm 1 with the
    same exhaustive fallback) pick the same 3-vertex part on every connected graph."""
    import oracle
    pairs = [(i, j) for i in range(k) for j in range(i + 1, k)]
    ids = list(range(k))
    for mask in range(1 << len(pairs)):
        rows = [0] * k
        for q, (a, b) in enumerate(pairs):
            if mask >> q & 1:
                rows[a] |= 1 << b
                rows[b] |= 1 << a
        if not _connected(k, rows):
            continue
        lm, _, _ = fsm.fsm_debug_dissect(ids, rows)
        assert oracle.dissect(rows) == lm, (k, rows)
