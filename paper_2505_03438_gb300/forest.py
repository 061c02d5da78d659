"""Random-forest classifier of the Random Forest tuning strategy (Sec. 5.3).

The paper trains a random-forest classifier (100 trees) whose features are
the live statistics of Sec. 4 and whose class is the configuration that
performed best on a synthetic scenario; during a simulation the forest
suggests the configuration to use.  Here the forest is trained by this
module (CART trees, Gini impurity, bootstrap samples, a random subset of
about sqrt(features) features tried at each split), stored as JSON in the
flattened layout of `ljsel_forest`, and evaluated inside the library
(`ljsel_forest_predict`, strategy 3 of `ljsel_autotune`).

Training data: one record per scenario, `{"name", "features": [8 floats],
"costs": {configuration name: ms per step}}`, as written by
`paper_2505_03438_gb300.forest_data` (a full search per scenario on the
GPU).  The class of a record is its cheapest configuration.

    python -m paper_2505_03438_gb300.forest DATA.jsonl MODEL.json
"""
import json
import math
import os
import sys

import numpy as np

FEATURES = ("mean", "rel_std", "median", "max", "nbins", "nempty", "skin", "threads")
HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_DATA = os.path.join(HERE, "forest_data.jsonl")
DEFAULT_MODEL = os.path.join(HERE, "forest_model.json")


def _gini_split(x, y, ncls):
    """Best threshold on one feature: (weighted child impurity, threshold),
    or None when the feature is constant.  Splits lie midway between
    consecutive distinct values; left is x <= threshold."""
    order = np.argsort(x, kind="stable")
    xs, ys = x[order], y[order]
    n = len(xs)
    onehot = np.zeros((n, ncls))
    onehot[np.arange(n), ys] = 1.0
    left = np.cumsum(onehot, axis=0)[:-1]          # class counts of the first k+1 samples
    right = left[-1] + onehot[-1] - left
    nl = np.arange(1, n, dtype=np.float64)
    nr = n - nl
    gl = 1.0 - ((left / nl[:, None]) ** 2).sum(1)
    gr = 1.0 - ((right / nr[:, None]) ** 2).sum(1)
    imp = (nl * gl + nr * gr) / n
    ok = xs[1:] > xs[:-1]
    if not ok.any():
        return None
    imp = np.where(ok, imp, np.inf)
    k = int(np.argmin(imp))
    return float(imp[k]), 0.5 * (float(xs[k]) + float(xs[k + 1]))


def _grow(X, y, ncls, rng, mtry, max_depth, nodes):
    """Grow one tree over the samples (X, y) depth first; append its nodes to
    `nodes` (dicts) and return the index of its root."""
    def build(idx, depth):
        counts = np.bincount(y[idx], minlength=ncls).astype(np.float64)
        me = len(nodes)
        nodes.append(None)
        gini = 1.0 - ((counts / counts.sum()) ** 2).sum()
        best = None
        if depth < max_depth and len(idx) >= 2 and counts.max() < len(idx):
            for f in rng.choice(X.shape[1], size=mtry, replace=False):
                s = _gini_split(X[idx, f], y[idx], ncls)
                if s is not None and s[0] < gini - 1e-12 and (best is None or s[0] < best[0]):
                    best = (s[0], int(f), s[1])
        if best is None:
            nodes[me] = dict(feature=-1, threshold=0.0, left=-1, right=-1, value=(counts / counts.sum()).tolist())
            return me
        _, f, thr = best
        go_left = X[idx, f] <= thr
        li = build(idx[go_left], depth + 1)
        ri = build(idx[~go_left], depth + 1)
        nodes[me] = dict(feature=f, threshold=thr, left=li, right=ri, value=[0.0] * ncls)
        return me

    return build(np.arange(len(y)), 0)


def train(X, labels, ntrees=100, max_depth=12, seed=0):
    """Random forest over features X (n x nfeatures) and class names
    `labels`; returns the model dict (the ljsel_forest arrays, classes by
    name)."""
    X = np.asarray(X, np.float64)
    classes = sorted(set(labels))
    y = np.array([classes.index(c) for c in labels], np.int64)
    ncls, nfeat = len(classes), X.shape[1]
    mtry = max(1, int(round(math.sqrt(nfeat))))
    rng = np.random.default_rng(seed)
    nodes, roots = [], []
    for _ in range(ntrees):
        boot = rng.integers(0, len(y), len(y))
        roots.append(_grow(X[boot], y[boot], ncls, rng, mtry, max_depth, nodes))
    return dict(nfeatures=nfeat, classes=classes, root=roots,
                feature=[n["feature"] for n in nodes], threshold=[n["threshold"] for n in nodes],
                left=[n["left"] for n in nodes], right=[n["right"] for n in nodes],
                value=[v for n in nodes for v in n["value"]])


def predict_proba(model, x):
    """Class probabilities for one feature vector: the mean over the trees of
    the leaf distributions (trees summed in order, as the library does)."""
    ncls = len(model["classes"])
    feat, thr, left, right, val = (model[k] for k in ("feature", "threshold", "left", "right", "value"))
    p = np.zeros(ncls)
    for r in model["root"]:
        k = r
        while feat[k] >= 0:
            k = left[k] if x[feat[k]] <= thr[k] else right[k]
        p += np.asarray(val[k * ncls:(k + 1) * ncls])
    return p / len(model["root"])


def records(path=DEFAULT_DATA):
    with open(path) as f:
        return [json.loads(line) for line in f if line.strip()]


def labelled(recs):
    """(features, cheapest configuration) of every record."""
    X = [r["features"] for r in recs]
    y = [min(r["costs"].items(), key=lambda kv: kv[1])[0] for r in recs]
    return X, y


def save(model, path=DEFAULT_MODEL):
    with open(path, "w") as f:
        json.dump(model, f)


def load(path=DEFAULT_MODEL):
    with open(path) as f:
        return json.load(f)


def main(argv):
    data = argv[1] if len(argv) > 1 else DEFAULT_DATA
    out = argv[2] if len(argv) > 2 else DEFAULT_MODEL
    X, y = labelled(records(data))
    model = train(X, y)
    save(model, out)
    print("%d records, %d classes, %d nodes -> %s" % (len(y), len(model["classes"]), len(model["feature"]), out))


if __name__ == "__main__":
    main(sys.argv)
