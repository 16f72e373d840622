"""Sampled mining and the support-prediction network on the GPU.

* The sampled last level against the oracle: an embedding is kept iff the 3-vertex part of its
  smallest-vertex-first dissection passes the splitmix64 rule; for every exactly frequent
  pattern (all of whose embeddings the GPU generates) the sampled MNI support and embedding
  count agree exactly, and for the other candidates the GPU's (pruned) values never exceed
  the oracle's.
* The network's forward pass, gradient and Adam step against the float64 reference
  (oracle/mlp.py), with the GPU's BF16-rounded weights.
* Sampled mining with a trained network: exactly recounted supports are exact, and the
  network's decisions beat the plain estimator on held-out graphs.
"""
import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle
import oracle.mlp as ref

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


def _keys(res, k):
    return [tuple(int(x) for x in l) + (int(a),) for l, a in zip(res["labels"], res["adj"])]


@pytest.mark.parametrize("case", [("er1000", 3, 10, 0.25), ("er1000", 4, 10, 0.25), ("er1000", 5, 10, 0.5),
                                  ("cl", 4, 5, 0.1), ("cl", 4, 5, 0.5)])
def test_sampled_candidates_match_oracle(fsm, case):
    name, k, t, p = case
    g = gg.workload("er1000") if name == "er1000" else gg.workload("cl100k", scale=0.005, cap=30)
    seed = 12345
    G = fsm.Graph.from_graphgen(g)
    G.set_option("candidates", 1)
    G.set_option("seed", seed)
    got = G.mine(k, t, sample_rate=p, features=True, stats=True)
    G.close()
    o = oracle.mine(g, k, 1, sample=(p, seed))
    okeys = {q: i for i, q in enumerate(_keys(o, k))}
    checked = 0
    for i, q in enumerate(_keys(got, k)):
        j = okeys[q]
        est_s = int(np.rint(o["ssupport"][j] / p))
        est_c = int(np.rint(o["scount"][j] / p))
        if o["support"][j] >= t:
            assert (int(got["support"][i]), int(got["count"][i])) == (est_s, est_c), q
            checked += 1
        else:
            assert got["support"][i] <= est_s and got["count"][i] <= est_c, q
    # every exactly frequent pattern with a kept embedding is a candidate
    cand = set(_keys(got, k))
    for q, j in okeys.items():
        if o["support"][j] >= t and o["scount"][j] > 0:
            assert q in cand, q
    assert checked > 0
    assert np.all(got["exact"] == 0)
    assert got["features"].shape == (len(got["support"]), 32) and np.all(np.isfinite(got["features"]))
    # the 32 features of every exactly frequent candidate, element by element, from the oracle's
    # sampled image sets (integer-derived entries exactly, the others within float32 rounding)
    cls = np.bincount(g.labels, minlength=g.num_labels)
    nfeat = 0
    for i, q in enumerate(_keys(got, k)):
        j = okeys[q]
        if o["support"][j] < t:
            continue
        f = got["features"][i].astype(np.float64)
        lab = [int(x) for x in o["labels"][j]]
        edges = oracle.pattern_edges(o["adj"][j], k)
        orbits, aut = _orbits(k, lab, edges)
        pop = o["spop"][j]
        for orb in orbits:
            assert len({int(pop[c]) for c in orb}) == 1, (q, orb, pop)
        pcs = sorted(int(pop[orb[0]]) for orb in orbits)
        assert [int(round(np.expm1(x))) for x in f[:len(pcs)]] == pcs, q
        assert np.all(f[len(pcs):8] == 0)
        tol = dict(rtol=1e-4, atol=1e-4)
        assert np.allclose(f[8:8 + k], [np.log(cls[l] / g.n) for l in lab], **tol) and np.all(f[8 + k:16] == 0)
        mean_deg = [o["sdeg"][j][c] / pop[c] if pop[c] else 0.0 for c in range(k)]
        assert np.allclose(f[16:16 + k], mean_deg, **tol) and np.all(f[16 + k:24] == 0), q
        assert f[24] == k and f[25] == len(edges)
        assert int(round(np.expm1(f[27]))) == int(o["scount"][j])
        assert int(round(np.exp(f[29]))) == aut
        assert np.allclose(f[[26, 28, 30, 31]], [np.log(p), np.log(t / g.n), np.log((min(pcs) + 1) / p), np.log(g.n)],
                           **tol)
        nfeat += 1
    assert nfeat == checked


def _orbits(k, lab, edges):
    """Orbits of a pattern's positions under its label-preserving automorphisms, and their
    number, by trying every permutation."""
    es = {frozenset(e) for e in edges}
    auts = [f for f in itertools.permutations(range(k))
            if all(lab[c] == lab[f[c]] for c in range(k)) and all(frozenset((f[a], f[b])) in es for a, b in edges)]
    seen, orbits = set(), []
    for c in range(k):
        if c in seen:
            continue
        orb = sorted({f[c] for f in auts})
        seen.update(orb)
        orbits.append(orb)
    return orbits, len(auts)


def _random_net(fsm, seed):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.25, ref.NPARAM).astype(np.float32)
    mean = rng.normal(0, 1, 32).astype(np.float32)
    sd = rng.uniform(0.5, 2, 32).astype(np.float32)
    m = fsm.fsm_mlp_create(seed)
    fsm.fsm_mlp_set_params(m, theta)
    fsm.fsm_mlp_set_norm(m, mean, sd)
    X = rng.normal(0, 2, (777, 32)).astype(np.float32)
    Y = rng.normal(0, 1, 777).astype(np.float32)
    return m, theta, mean, sd, X, Y


def test_mlp_forward_and_gradient_match_reference(fsm):
    m, theta, mean, sd, X, Y = _random_net(fsm, 3)
    try:
        p = ref.gpu_weights(theta)
        y_ref, _ = ref.forward(p, X, mean.astype(np.float64), sd.astype(np.float64))
        y_gpu = fsm.fsm_mlp_predict(m, X)
        # FP32 accumulation of <= 64-term products of BF16 weights and FP32 activations
        assert np.allclose(y_gpu, y_ref, rtol=1e-4, atol=1e-4)
        loss_ref, g_ref = ref.loss_and_grad(p, X, Y, mean.astype(np.float64), sd.astype(np.float64))
        g_gpu, loss_gpu = fsm.fsm_mlp_gradients(m, X, Y)
        assert abs(loss_gpu - loss_ref) <= 1e-4 * max(1.0, loss_ref)
        assert np.allclose(g_gpu, g_ref, rtol=1e-3, atol=1e-5 * max(1.0, float(np.abs(g_ref).max())))
    finally:
        fsm.fsm_mlp_free(m)


def test_adam_step_matches_reference(fsm):
    m, theta, mean, sd, X, Y = _random_net(fsm, 5)
    try:
        p = ref.gpu_weights(theta)
        _, g = ref.loss_and_grad(p, X, Y, mean.astype(np.float64), sd.astype(np.float64))
        th_ref, _, _ = ref.adam_step(theta.astype(np.float64), np.zeros(ref.NPARAM), np.zeros(ref.NPARAM), g, 1, 1e-3)
        fsm.fsm_mlp_train(m, X, Y, epochs=1, batch=len(Y), lr=1e-3, seed=0)
        th_gpu = fsm.fsm_mlp_get_params(m)
        # the first Adam step moves each weight by about lr * sign(g); compare the moves
        assert np.allclose(th_gpu - theta, th_ref - theta, atol=2e-5)
    finally:
        fsm.fsm_mlp_free(m)


def test_training_fits_a_smooth_function(fsm):
    rng = np.random.default_rng(9)
    X = rng.normal(0, 1, (4096, 32)).astype(np.float32)
    Y = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2]).astype(np.float32)
    m = fsm.fsm_mlp_create(1)
    try:
        fsm.fsm_mlp_set_norm(m, np.zeros(32), np.ones(32))
        _, l0 = fsm.fsm_mlp_gradients(m, X, Y)
        l1 = fsm.fsm_mlp_train(m, X, Y, epochs=60, batch=128, lr=3e-3, seed=2)
        assert l1 < 0.2 * l0
    finally:
        fsm.fsm_mlp_free(m)


def test_learned_sampling_recounts_exactly_and_beats_the_plain_estimator(fsm):
    from paper_2101_07690_gb300 import learn
    k, p = 4, 0.1
    train = [gg.workload("cl100k", scale=0.03, cap=60, seed=s) for s in range(10, 16)]
    held = [gg.workload("cl100k", scale=0.03, cap=60, seed=s) for s in (40, 41)]
    t = 30
    Xs, ys = [], []
    for g in train:
        X, y, _ = learn.training_pairs(g, k, t, p, seed=1)
        Xs.append(X)
        ys.append(y)
    X, y = np.concatenate(Xs), np.concatenate(ys)
    m = learn.fit(X, y, epochs=200, batch=256, lr=3e-3, seed=0)
    try:
        stats = {"model": [], "plain": []}
        for g in held:
            G = fsm.Graph.from_graphgen(g)
            exact = learn.frequent_set(G.mine(k, t), k)
            G.set_option("seed", 1)
            plain = G.mine(k, t, sample_rate=p)
            G.set_option("model", m)
            G.set_option("delta_milli", 700)
            learned = G.mine(k, t, sample_rate=p)
            G.close()
            # exactly recounted supports and counts are the oracle's (its one-pattern matcher,
            # on up to 150 recounted patterns, the smallest supports first)
            rec = [(int(s), i) for i, (s, e) in enumerate(zip(learned["support"], learned["exact"])) if e]
            for s_, i in sorted(rec)[:150]:
                sup, cnt = oracle.pattern_support(g, learned["labels"][i], int(learned["adj"][i]))
                assert (sup, cnt) == (s_, int(learned["count"][i]))
                assert exact.get(_keys(learned, k)[i]) == s_
            stats["model"].append(learn.compare(exact, learn.frequent_set(learned, k)))
            stats["plain"].append(learn.compare(exact, learn.frequent_set(plain, k)))
        rec_m = np.mean([s["recall"] for s in stats["model"]])
        rec_p = np.mean([s["recall"] for s in stats["plain"]])
        f1 = lambda s: 2 * s["precision"] * s["recall"] / max(s["precision"] + s["recall"], 1e-9)
        f1_m = np.mean([f1(s) for s in stats["model"]])
        f1_p = np.mean([f1(s) for s in stats["plain"]])
        print("learned", stats["model"], "plain", stats["plain"])
        assert f1_m >= f1_p and rec_m >= rec_p
    finally:
        fsm.fsm_mlp_free(m)


def test_fit_norm_matches_the_standardisation_of_the_data(fsm):
    """fsm_mlp_fit_norm computes the input means and (population) standard deviations on the
    device, floored at 1e-3: predictions equal those of a network given numpy's."""
    rng = np.random.default_rng(12)
    X = rng.normal(3.0, 2.0, (5000, 32)).astype(np.float32)
    X[:, 7] = 1.5   # a constant column: deviation floored
    theta = rng.normal(0, 0.25, ref.NPARAM).astype(np.float32)
    a, b = fsm.fsm_mlp_create(1), fsm.fsm_mlp_create(1)
    try:
        for m in (a, b):
            fsm.fsm_mlp_set_params(m, theta)
        fsm.fsm_mlp_fit_norm(a, X)
        x64 = X.astype(np.float64)
        fsm.fsm_mlp_set_norm(b, x64.mean(axis=0), np.maximum(x64.std(axis=0), 1e-3))
        assert np.allclose(fsm.fsm_mlp_predict(a, X), fsm.fsm_mlp_predict(b, X), rtol=1e-4, atol=1e-4)
    finally:
        fsm.fsm_mlp_free(a)
        fsm.fsm_mlp_free(b)
