"""Training and evaluation harness of the support-prediction network of sampled mining.

Training pairs come from the library itself: on each seeded training graph, sampled mining
with option "candidates" gives every candidate pattern's 32 features, and exact mining at
threshold 1 gives every pattern's exact MNI support; pairs are joined by canonical code and the
target is log(support).  Fitting, prediction and all network arithmetic run in the library's
CUDA kernels (fsm_mlp_*); this module only moves arrays between calls.
"""
from __future__ import annotations

import numpy as np

from . import fsm


def _keys(res, k):
    return [tuple(int(x) for x in l) + (int(a),) for l, a in zip(res["labels"], res["adj"])]


def training_pairs(graph, k: int, t: int, p: float, seed: int = 0, mode: str = "edge", t_label: int = 1):
    """(features, log exact support, keys) of every candidate pattern of sampled mining.

    Exact supports come from exact mining at threshold t_label (1: every pattern).  For large k
    a t_label above 1 keeps that run tractable; a candidate whose exact support is below t_label
    then gets the censored target log(t_label / 2)."""
    G = fsm.Graph.from_graphgen(graph, mode)
    try:
        G.set_option("fused", 1)
        exact = G.mine(k, t_label)
        G.set_option("fused", 0)
        G.set_option("candidates", 1)
        G.set_option("seed", seed)
        cand = G.mine(k, t, sample_rate=p, features=True)
    finally:
        G.close()
    sup = dict(zip(_keys(exact, k), exact["support"]))
    keys = _keys(cand, k)
    low = max(1.0, t_label / 2.0)
    y = np.array([np.log(float(sup.get(q, low))) for q in keys], np.float32)
    return cand["features"].astype(np.float32), y, keys


def fit(X, y, epochs: int = 300, batch: int = 256, lr: float = 3e-3, seed: int = 0):
    """A trained network handle (free with fsm.fsm_mlp_free)."""
    m = fsm.fsm_mlp_create(seed)
    fsm.fsm_mlp_fit_norm(m, X)   # input standardisation, computed by the library
    fsm.fsm_mlp_train(m, X, y, epochs, batch, lr, seed)
    return m


def frequent_set(res, k):
    return {q: int(s) for q, s in zip(_keys(res, k), res["support"])}


def compare(exact: dict, got: dict) -> dict:
    """Precision and recall of the frequent set and the median relative support error over
    the true positives."""
    tp = [q for q in got if q in exact]
    prec = len(tp) / len(got) if got else 1.0
    rec = len(tp) / len(exact) if exact else 1.0
    err = [abs(got[q] - exact[q]) / exact[q] for q in tp]
    return {"precision": prec, "recall": rec, "median_rel_err": float(np.median(err)) if err else 0.0,
            "exact_patterns": len(exact), "returned": len(got)}


def quota_rows(G, k: int, t: int, exact: dict, quotas, seed: int = 1) -> list:
    """Section 5's own sampling (ST x: x^2 candidate pieces per key group, x edges per key vertex
    when edges are joined) on an open graph handle, for each x: time, and precision, recall and
    median support error against the exact frequent set.  The drawn supports are lower bounds,
    so precision is 1 by construction."""
    import sys
    import time
    rows = []
    G.set_option("model", 0)
    G.set_option("seed", seed)
    for x in quotas:
        G.set_option("join_quota", int(x))
        t0 = time.perf_counter()
        r = G.mine(k, t)
        row = {"join_quota": int(x), "seconds": time.perf_counter() - t0}
        row.update(compare(exact, frequent_set(r, k)))
        rows.append(row)
        sys.stderr.write(f"[quota] {row}\n")
        sys.stderr.flush()
    G.set_option("join_quota", 0)
    return rows


def study(workload: str, k: int, t: int, p: float, train_scale: float, train_seeds, cap, test_scale: float = 1.0,
          test_cap=None, deltas=(0.0, 0.1, 0.25, 0.5), epochs: int = 200, seed: int = 1, quotas=(),
          label_frac: float = 0.0, max_pairs: int = 0) -> dict:
    """Train on copies of a workload (other seeds), then mine the test graph exactly, with the
    plain sampled estimator, with the learned decision plus exact recount for each recount band
    delta, and with Section 5's quotas ST x for each x in quotas; report time and accuracy of
    each against the exact result, and the network's error on held-out training pairs."""
    import sys
    import time

    import graphgen as gg

    t_start = time.perf_counter()

    def note(msg):   # progress on stderr, so a run cut short still shows how far it got
        sys.stderr.write(f"[study {time.perf_counter() - t_start:8.1f} s] {msg}\n")
        sys.stderr.flush()

    test = gg.workload(workload, scale=test_scale, cap=test_cap)
    Xs, ys = [], []
    for s in train_seeds:
        g = gg.workload(workload, scale=train_scale, cap=cap, seed=s)
        # the same threshold relative to the graph size (the paper's thresholds are fractions of n)
        tt = max(1, int(round(t * g.n / test.n)))
        X, y, _ = training_pairs(g, k, tt, p, seed=seed, t_label=max(1, int(round(tt * label_frac))))
        Xs.append(X)
        ys.append(y)
        note(f"training graph seed {s}: n={g.n} t={tt}, {len(y)} pairs")
    X, y = np.concatenate(Xs), np.concatenate(ys)
    rng = np.random.default_rng(seed)
    if max_pairs and len(y) > max_pairs:   # large k: millions of candidates; train on a uniform subsample
        pick = rng.choice(len(y), size=max_pairs, replace=False)
        X, y = X[pick], y[pick]
        note(f"training on a uniform subsample of {max_pairs} pairs")
    perm = rng.permutation(len(y))
    nval = len(y) // 10
    val, tr = perm[:nval], perm[nval:]
    m = fit(X[tr], y[tr], epochs=epochs, seed=seed)
    try:
        err = fsm.fsm_mlp_predict(m, X[val]) - y[val]
        out = {"train_pairs": int(len(tr)), "val_rmse_log": float(np.sqrt(np.mean(err ** 2))),
               "val_median_abs_log_err": float(np.median(np.abs(err))),
               "test_n": test.n, "test_m": test.m, "k": k, "t": t, "p": p}
        G = fsm.Graph.from_graphgen(test)
        G.set_option("launch", 1)
        G.set_option("fused", 1)
        G.mine(k, t)   # first call: lazy set-up and autotuning
        t0 = time.perf_counter()
        exact = frequent_set(G.mine(k, t), k)
        out["exact_s"] = time.perf_counter() - t0
        G.set_option("fused", 0)
        note(f"exact: {out['exact_s']:.1f} s, {len(exact)} frequent patterns")
        G.set_option("seed", seed)
        t0 = time.perf_counter()
        plain = frequent_set(G.mine(k, t, sample_rate=p), k)
        out["plain_s"] = time.perf_counter() - t0
        out["plain"] = compare(exact, plain)
        note(f"plain estimator: {out['plain_s']:.1f} s {out['plain']}")
        G.set_option("model", m)
        out["learned"] = []
        for delta in deltas:
            G.set_option("delta_milli", int(delta * 1000))
            t0 = time.perf_counter()
            r = G.mine(k, t, sample_rate=p, stats=True)
            row = {"delta": delta, "seconds": time.perf_counter() - t0,
                   "recounted": int(r["stats"]["recount_patterns"]), "exactly_counted": int(r["exact"].sum())}
            row.update(compare(exact, frequent_set(r, k)))
            out["learned"].append(row)
            note(f"learned: {row}")
        G.set_option("delta_milli", 500)
        if quotas:
            out["quota"] = quota_rows(G, k, t, exact, quotas, seed=seed)
        G.close()
        return out
    finally:
        fsm.fsm_mlp_free(m)


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="learned sampled mining study")
    ap.add_argument("--workload", default="cl100k")
    ap.add_argument("--k", type=int, default=5)
    ap.add_argument("--t", type=int, default=1000)
    ap.add_argument("--p", type=float, default=0.05)
    ap.add_argument("--train-scale", type=float, default=1.0)
    ap.add_argument("--train-seeds", default="10-13")
    ap.add_argument("--cap", type=float, default=300)
    ap.add_argument("--test-cap", type=float, default=300)
    ap.add_argument("--deltas", default="0,0.05,0.1,0.25,0.5")
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--quotas", default="", help="Section 5 ST x values to compare, e.g. 2,4,8")
    ap.add_argument("--test-scale", type=float, default=1.0)
    ap.add_argument("--label-frac", type=float, default=0.0,
                    help="exact training labels from mining at this fraction of the threshold (0: threshold 1)")
    ap.add_argument("--max-pairs", type=int, default=0, help="train on at most this many (uniformly drawn) pairs")
    a = ap.parse_args()
    lo, hi = (int(x) for x in a.train_seeds.split("-"))
    print(json.dumps(study(a.workload, a.k, a.t, a.p, a.train_scale, range(lo, hi + 1), a.cap,
                           test_scale=a.test_scale, test_cap=a.test_cap, deltas=[float(x) for x in a.deltas.split(",")],
                           epochs=a.epochs, quotas=[int(x) for x in a.quotas.split(",") if x],
                           label_frac=a.label_frac, max_pairs=a.max_pairs)))
