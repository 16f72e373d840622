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


def training_pairs(graph, k: int, t: int, p: float, seed: int = 0, mode: str = "edge"):
    """(features, log exact support, keys) of every candidate pattern of sampled mining."""
    G = fsm.Graph.from_graphgen(graph, mode)
    try:
        exact = G.mine(k, 1)
        G.set_option("candidates", 1)
        G.set_option("seed", seed)
        cand = G.mine(k, t, sample_rate=p, features=True)
    finally:
        G.close()
    sup = dict(zip(_keys(exact, k), exact["support"]))
    keys = _keys(cand, k)
    y = np.array([np.log(float(sup[q])) for q in keys], np.float32)
    return cand["features"].astype(np.float32), y, keys


def fit(X, y, epochs: int = 300, batch: int = 256, lr: float = 3e-3, seed: int = 0):
    """A trained network handle (free with fsm.fsm_mlp_free)."""
    m = fsm.fsm_mlp_create(seed)
    mean = X.mean(axis=0)
    sd = np.maximum(X.std(axis=0), 1e-3)
    fsm.fsm_mlp_set_norm(m, mean, sd)
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
