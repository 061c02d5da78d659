"""The Predictive strategy's trial rule (Sec. 5.1) as host logic, through
the C-ABI, without a GPU: the first two phases trial everything; later a
configuration is trialled when its cost, extrapolated along the line
through its last two measurements, is within the factor of the best
prediction, when it is stale, unmeasured, or the incumbent; blacklisted
configurations never are."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lj():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_03438_gb300 as m
    return m


def test_first_two_phases_trial_everything_but_the_blacklist(lj):
    hist = [[(0, 5.0)], [], [(0, 0.1)]]
    for phase in (0, 1):
        assert lj.ljsel_predictive_trials(phase, hist, [0, -1, 0], [0, 0, 1]) == [1, 1, 0]


def test_linear_extrapolation_and_the_factor(lj):
    # A: 1.0 at phase 0, 2.0 at phase 1 -> predicted 3.0 at phase 2, 4.0 at phase 3
    # B: one measurement, 1.5 -> predicted 1.5; factor 2 -> threshold 3.0
    hist = [[(0, 1.0), (1, 2.0)], [(1, 1.5)]]
    assert lj.ljsel_predictive_trials(2, hist, [1, 1], [0, 0]) == [1, 1]  # 3.0 <= 3.0
    assert lj.ljsel_predictive_trials(3, hist, [1, 1], [0, 0]) == [0, 1]  # 4.0 > 3.0
    # only the last two measurements count
    hist3 = [[(0, 50.0), (1, 1.0), (2, 2.0)], [(2, 1.5)]]
    assert lj.ljsel_predictive_trials(4, hist3, [2, 2], [0, 0]) == [0, 1]  # 4.0 > 3.0
    assert lj.ljsel_predictive_trials(3, hist3, [2, 2], [0, 0]) == [1, 1]  # 3.0 <= 3.0
    # a wider factor lets A in
    assert lj.ljsel_predictive_trials(3, hist, [1, 1], [0, 0], predict_factor=3.0) == [1, 1]


def test_a_steep_fall_cannot_exclude_everything_else(lj):
    # A fell from 10 to 2 between two phases: the line predicts -6 at phase 2;
    # the prediction is held at half of the last measurement (1.0), so B
    # (0.3) stays the expected optimum and A is not trialled
    hist = [[(0, 10.0), (1, 2.0)], [(0, 0.3), (1, 0.3)], [(0, 0.35), (1, 0.32)]]
    assert lj.ljsel_predictive_trials(2, hist, [1, 1, 1], [0, 0, 0]) == [0, 1, 1]


def test_incumbent_stale_unmeasured_and_blacklisted(lj):
    hist = [[(0, 0.2), (1, 0.2)], [(0, 5.0), (1, 5.0)], [(0, 5.0), (1, 5.0)], [], [(0, 0.1), (1, 0.1)]]
    last = [1, 1, 1, -1, 1]
    bl = [0, 0, 0, 0, 1]
    # the slow configuration 1 is the incumbent: trialled; 2 is not
    assert lj.ljsel_predictive_trials(2, hist, last, bl, incumbent=1) == [1, 1, 0, 1, 0]
    # configuration 2 last trialled 4 phases ago: stale, retrialled
    last2 = [5, 5, 1, -1, 5]
    assert lj.ljsel_predictive_trials(5, hist, last2, bl, retrial_phases=4) == [1, 0, 1, 1, 0]
    assert lj.ljsel_predictive_trials(5, hist, last2, bl, retrial_phases=5) == [1, 0, 0, 1, 0]
    # the blacklist wins over everything, the incumbent included
    assert lj.ljsel_predictive_trials(2, hist, last, bl, incumbent=4) == [1, 0, 0, 1, 0]


def test_invalid_arguments(lj):
    L = lj.lib()
    n = 2
    hn = np.array([1, 3], np.int32)
    hp = np.zeros(4, np.int32)
    hc = np.ones(4)
    lt = np.zeros(2, np.int32)
    bl = np.zeros(2, np.int32)
    out = np.zeros(2, np.int32)
    args = lambda hn_, inc, f: (n, 2, hn_.ctypes.data, hp.ctypes.data, hc.ctypes.data, lt.ctypes.data, bl.ctypes.data,
                                inc, f, 4, out.ctypes.data)
    assert L.ljsel_predictive_trials(*args(hn, -1, 2.0)) == 1  # hist_n = 3
    hn[1] = 1
    assert L.ljsel_predictive_trials(*args(hn, 2, 2.0)) == 1  # incumbent out of range
    assert L.ljsel_predictive_trials(*args(hn, -1, 0.0)) == 1  # factor <= 0
    assert L.ljsel_predictive_trials(-1, 2, None, None, None, None, None, -1, 2.0, 4, None) == 1
    assert L.ljsel_predictive_trials(2, 2, None, None, None, None, None, -1, 2.0, 4, None) == 1
    assert L.ljsel_predictive_trials(0, 2, None, None, None, None, None, -1, 2.0, 4, None) == 0
    assert L.ljsel_predictive_trials(*args(hn, 1, 2.0)) == 0
