"""The random forest of the Random Forest strategy (Sec. 5.3), host only:
training (CART, Gini) on data whose rule is known, the library's
evaluation of a forest against the numpy one bit for bit, rejection of
malformed forests, and the shipped model being the one its shipped data
and the training code produce."""
import numpy as np
import pytest

from paper_2505_03438_gb300 import forest

NAMES = ["VL-noN3L-t2-R10-csf1", "LC-N3L-t1-R10-csf1", "VLW-noN3L-t1-R10-csf1"]


@pytest.fixture(scope="module")
def lj():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_03438_gb300 as m
    return m


def _rule(X):
    return [NAMES[0] if x[0] > 5 else (NAMES[1] if x[3] > 4 else NAMES[2]) for x in X]


def test_gini_split_by_hand():
    # x: 1 2 3 4, classes 0 0 1 1: the split at 2.5 leaves both sides pure
    imp, thr = forest._gini_split(np.array([3.0, 1.0, 4.0, 2.0]), np.array([1, 0, 1, 0]), 2)
    assert thr == 2.5 and imp == 0.0
    # classes 0 1 0 1 over 1 2 3 4: best is after the first sample (3 left
    # of 1 right is symmetric): left {0}, right {1,0,1}: (1*0 + 3*(1-(1/9+4/9)))/4
    imp, thr = forest._gini_split(np.array([1.0, 2.0, 3.0, 4.0]), np.array([0, 1, 0, 1]), 2)
    assert thr in (1.5, 3.5) and abs(imp - 3 * (1 - 5 / 9) / 4) < 1e-15
    # constant feature: no split
    assert forest._gini_split(np.ones(5), np.array([0, 1, 0, 1, 0]), 2) is None


def test_training_recovers_a_known_rule():
    rng = np.random.default_rng(0)
    X = rng.uniform(0, 10, (300, 8))
    m = forest.train(X, _rule(X), ntrees=30, seed=1)
    Xt = rng.uniform(0, 10, (300, 8))
    pred = [m["classes"][int(np.argmax(forest.predict_proba(m, x)))] for x in Xt]
    assert np.mean([a == b for a, b in zip(pred, _rule(Xt))]) >= 0.95
    # leaf distributions are probabilities, and so is the forest's output
    p = forest.predict_proba(m, Xt[0])
    assert abs(p.sum() - 1.0) < 1e-12 and (p >= 0).all()


def test_library_evaluates_forests_as_numpy_does(lj):
    rng = np.random.default_rng(2)
    X = rng.uniform(0, 10, (200, 8))
    models = [forest.train(X, _rule(X), ntrees=20, seed=3), forest.load()]
    for m in models:
        for x in rng.uniform(-5, 50, (100, 8)):
            assert np.array_equal(lj.ljsel_forest_predict(m, x), forest.predict_proba(m, x))
        # a feature exactly on a split threshold goes left (x <= threshold)
        for r in m["root"]:
            f = m["feature"][r]
            if f < 0:
                continue
            x = np.zeros(8)
            x[f] = m["threshold"][r]
            assert np.array_equal(lj.ljsel_forest_predict(m, x), forest.predict_proba(m, x))
    # the shipped model on its own training features
    m = forest.load()
    for r in forest.records():
        assert np.array_equal(lj.ljsel_forest_predict(m, r["features"]), forest.predict_proba(m, r["features"]))


def _malformed(m, **edits):
    bad = {k: (list(v) if isinstance(v, list) else v) for k, v in m.items()}
    for k, (i, val) in edits.items():
        bad[k][i] = val
    return bad


def test_malformed_forests_are_rejected(lj):
    rng = np.random.default_rng(4)
    X = rng.uniform(0, 10, (60, 8))
    m = forest.train(X, _rule(X), ntrees=3, seed=5)
    nn = len(m["feature"])
    split = next(k for k in range(nn) if m["feature"][k] >= 0)
    leaf = next(k for k in range(nn) if m["feature"][k] < 0)
    cases = [
        _malformed(m, root=(0, nn)),                      # root out of range
        _malformed(m, left=(split, nn)),                  # child out of range
        _malformed(m, right=(split, -1)),
        _malformed(m, feature=(split, 8)),                # feature >= nfeatures
        _malformed(m, left=(split, split)),               # a cycle
        _malformed(m, value=(leaf * len(m["classes"]), -0.5)),  # negative leaf value
        _malformed(m, threshold=(split, float("nan"))),
        dict(m, nfeatures=9),
    ]
    assert split == 0  # the first tree's root splits; x = -1e9 goes left there
    for bad in cases:
        with pytest.raises(lj.LjselError) as e:
            lj.ljsel_forest_predict(bad, np.full(8, -1e9))
        assert e.value.status == 1  # LJSEL_ERR_ARG


def test_shipped_model_is_reproducible_from_shipped_data():
    X, y = forest.labelled(forest.records())
    assert len(y) >= 40 and len(X[0]) == len(forest.FEATURES)
    assert forest.train(X, y) == forest.load()
    # every record's class is its cheapest configuration
    for r, c in zip(forest.records(), y):
        assert r["costs"][c] == min(r["costs"].values())


def test_training_scenarios_are_physical_inputs():
    """The forest's training scenarios (input generators only): every particle
    inside its box, no two closer than the 0.9 spacing outside the jittered
    lattices (whose nearest neighbours sit at a/sqrt(2) - 0.1*sqrt(3) or
    more), zero momentum and the drawn temperature exactly, boxes that admit
    the minimum image at the scenario's skin, skins cycling 0.1 ... 0.5 (the
    walled spheres at the heating run's settings)."""
    from scipy.spatial import cKDTree

    from paper_2505_03438_gb300 import scenarios
    seen, walled = [], []
    for sc in scenarios.training_scenarios():
        x, v, L = sc["x"], sc["v"], sc["box"][0]
        n = len(x)
        assert (x >= 0).all() and (x < L).all(), sc["name"]
        assert L >= 2 * (2.5 + sc["skin"]) * (1 + 1 / 1024), sc["name"]
        if n > 1:
            d, _ = cKDTree(x, boxsize=L).query(x, k=2)
            floor = 0.9 if not sc["name"].startswith("fcc") else 0.8
            assert d[:, 1].min() >= floor - 1e-9, (sc["name"], d[:, 1].min())
            assert np.abs(v.sum(0)).max() < 1e-9 * n, sc["name"]
            assert abs((v * v).sum() / (3 * n - 3) - sc["temperature"]) < 1e-9, sc["name"]
        seen.append((sc["name"], sc["skin"]))
        if sc.get("walls"):
            assert sc["skin"] == 0.5 and sc["dt"] == 1e-4 and float(np.max(sc["rcut"])) == 3.0, sc["name"]
            walled.append((sc["name"], n, L))
    assert len(seen) == 49
    assert [s for _, s in seen[:10]] == [0.1, 0.2, 0.3, 0.4, 0.5] * 2
    # the benchmark workloads are not among them (the walled heating run is
    # 5497 particles in a box of 200)
    assert not any(nm.startswith("fcc_n64") or nm.startswith("heated") for nm, _ in seen)
    assert len(walled) == 7 and not any(n == 5497 for _, n, _ in walled)
