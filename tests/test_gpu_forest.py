"""The Random Forest strategy (Sec. 5.3) on the GPU with the shipped forest:
with forest_top 1 a phase selects the configuration the forest ranks first
for the live statistics (computed here from the same statistics with the
numpy forest) without a trial; with forest_top k > 1 it trials exactly the
k first-ranked configurations and keeps the cheapest; the trial steps
advance the simulation on the oracle's FP64 trajectory."""
import numpy as np
import pytest

import oracle
import paper_2505_03438_gb300 as lj
from paper_2505_03438_gb300 import forest, scenarios

pytestmark = pytest.mark.gpu


def _orc_params(sc):
    return oracle.make_params(sc["box"], sc["eps"], sc["sigma"], sc["rcut"], sc.get("shift", True))


def _wrapdiff(a, b, L):
    d = a - b
    return d - L * np.round(d / L)


def test_forest_strategy_trials_the_forests_first_choices():
    sc = scenarios.fcc_liquid(8, seed=71, jitter=0.1)
    s = lj.System(sc, precision=1)
    with pytest.raises(lj.LjselError) as e:
        s.autotune(strategy="forest")
    assert e.value.status == 8  # LJSEL_ERR_STATE: no forest installed
    m = forest.load()
    s.set_forest(m)
    trialled = selected = 0
    blacklist = set()  # configurations a trial measured 10x slower than the best (the default factor)
    for phase, top in enumerate((1, 1, 3, 2)):
        st = s.stats()
        p = forest.predict_proba(m, [st[k] for k in forest.FEATURES])
        ranked = [m["classes"][k] for k in np.argsort(-p, kind="stable")]
        expect = [nm for nm in ranked if nm not in blacklist][:top] if top > 1 else ranked[:1]
        before = s.config().name()
        c, rep = s.autotune(strategy="forest", trial_steps=4, forest_top=top)
        assert rep["expert_input"] == p.max() and rep["phase"] == phase + 1
        costs = {k: v for k, (v, ph) in lj.ljsel_tuner_costs(s.h).items() if ph == phase}
        if top == 1:
            # the single suggestion is selected without a trial
            assert rep["ntrialled"] == 0 and rep["trial_steps_total"] == 0 and not costs
            assert c.name() == expect[0] == s.config().name()
            selected += 1
            continue
        assert rep["ntrialled"] == top
        trialled += top
        assert sorted(costs) == sorted(expect)
        assert c.name() == min(costs, key=costs.get) and s.config().name() == c.name()
        best = min(costs.values())
        blacklist |= {nm for nm, v in costs.items() if v > 10.0 * best}
    assert selected == 2
    nsteps = s.counters()["steps"]
    assert nsteps == 4 * trialled
    x, v = s.state()
    xo, vo, *_ = oracle.verlet_run(sc["x"], sc["v"], None, [1.0], _orc_params(sc), sc["dt"], nsteps)
    assert np.abs(_wrapdiff(x, xo, sc["box"][0])).max() < 1e-9
    assert np.abs(v - vo).max() < 1e-9
    s.close()


def test_forest_classes_must_suit_the_system():
    sc = dict(scenarios.random_gas(300, 12.0, seed=72, min_dist=0.9), walls=(1, 1, 1))
    s = lj.System(sc)
    m = forest.train(np.random.default_rng(0).uniform(0, 1, (4, 8)), ["VLW-noN3L-t1-R10-csf1"] * 4, ntrees=2)
    with pytest.raises(lj.LjselError) as e:
        s.set_forest(m)  # window lists do not support walls
    assert e.value.status == 9  # LJSEL_ERR_UNSUPPORTED
    s.close()


def test_tuner_costs_cover_a_full_search():
    sc = scenarios.fcc_liquid(6, seed=73, jitter=0.1)
    s = lj.System(sc)
    cands = lj.ljsel_default_candidates(s.h)
    c, rep = s.autotune(strategy="full", trial_steps=3)
    costs = lj.ljsel_tuner_costs(s.h)
    assert sorted(costs) == sorted(k.name() for k in cands)
    assert all(v > 0 and ph == 0 for v, ph in costs.values())
    assert abs(costs[c.name()][0] - rep["chosen_cost_ms"]) < 1e-12
    s.close()
