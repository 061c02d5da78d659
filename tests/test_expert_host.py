"""The Expert strategy's fuzzy engine (Sec. 2.3 fuzzy logic, Sec. 5.2 Expert)
on the host, against centroids derived by hand.

Output sets on [0, 1]: bad = 1 on [0, 0.1] falling to 0 at 0.4; okay = the
triangle 0.2 / 0.5 / 0.8; good = 0 below 0.6 rising to 1 at 0.9.  Their
centres of gravity, with unit weight, integrated exactly:
  okay:  symmetric about 0.5                                    -> 0.5
  good:  area 0.15 + 0.1 = 0.25, moment 0.12 + 0.095 = 0.215    -> 0.86
  bad:   area 0.1 + 0.15 = 0.25, moment 0.005 + 0.03 = 0.035    -> 0.14
On the ramp at 2.5 particles per bin the input is half sparse, half medium
((4 - 2.5) / 3 and (2.5 - 1) / 3).  An okay and a good term, each clipped
at 0.5, aggregate to a set that rises on [0.2, 0.35], is 0.5 to 0.65,
follows okay down to the crossing at 0.7 (height 1/3), follows good up to
0.5 at 0.75 and stays there to 1.  Area 0.0375 + 0.15 + 0.0208333 +
0.0208333 + 0.125 = 0.3541667, moment 0.01125 + 0.075 + 0.0140278 +
0.0151389 + 0.109375 = 0.2247917, centroid 0.63471.  The library samples
the output at 201 points, which moves these values by at most 1.5e-3
(mostly the full-weight end samples at 0 and 1); the bar is 3e-3, far
below what a wrong term, rule or inference would cause (0.1 and more).
"""
import pytest

TOL = 3e-3


@pytest.fixture(scope="module")
def lj():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2505_03438_gb300 as m
    return m


def _cfg(lj, method):
    kw = {"CL": dict(cluster_size=4, threads_per_unit=4)}.get(method, {})
    return lj.make_config(method, **kw)


# (mean particles per bin, method) -> hand-derived centroid.  Rules
# (sparse / medium / dense): VL good / good / good, VLW and LC bad / bad /
# bad, CL bad / okay / okay.
PLATEAUS = [
    (0.0, "VL", 0.86), (0.0, "VLW", 0.14), (0.0, "LC", 0.14), (0.0, "CL", 0.14),
    (0.9, "LC", 0.14), (0.9, "CL", 0.14),
    (6.0, "VL", 0.86), (6.0, "VLW", 0.14), (6.0, "LC", 0.14), (6.0, "CL", 0.5),
    (12.0, "VL", 0.86), (19.1, "VLW", 0.14), (19.1, "LC", 0.14), (19.1, "CL", 0.5),
]


@pytest.mark.parametrize("x,method,expect", PLATEAUS, ids=lambda v: str(v))
def test_plateaus(lj, x, method, expect):
    assert abs(lj.ljsel_expert_suitability(_cfg(lj, method), x) - expect) < TOL


def _good_clipped_at_half():
    # good clipped at h = 0.5: 0 below 0.6, rising to h at 0.6 + 0.3 h, flat
    # to 1; its area and moment in closed form
    h = 0.5
    a = 0.3 * h
    area = 0.5 * a * h + (1.0 - 0.6 - a) * h
    # moment of the rising part: integral of y (y - 0.6) / 0.3 over [0.6, 0.6 + a]
    m_rise = ((0.6 + a) ** 3 / 3 - 0.3 * (0.6 + a) ** 2 - (0.6 ** 3 / 3 - 0.3 * 0.6 ** 2)) / 0.3
    m_flat = h * (1.0 - (0.6 + a) ** 2) / 2
    return (m_rise + m_flat) / area


def test_ramp_between_sparse_and_medium(lj):
    # at 2.5 the input is half sparse, half medium ((4 - 2.5) / 3 and
    # (2.5 - 1) / 3).  Cluster lists aggregate bad and okay, each clipped at
    # 0.5: the mirror image about 0.5 of the okay + good set of the header
    # (bad and good are mirror images, okay is symmetric)
    assert abs(lj.ljsel_expert_suitability(_cfg(lj, "CL"), 2.5) - (1.0 - 0.63471)) < TOL
    # Verlet lists: good from both terms, clipped at 0.5
    assert abs(lj.ljsel_expert_suitability(_cfg(lj, "VL"), 2.5) - _good_clipped_at_half()) < TOL
    # linked cells: bad from both terms, the mirror image of that
    assert abs(lj.ljsel_expert_suitability(_cfg(lj, "LC"), 2.5) - (1.0 - _good_clipped_at_half())) < TOL


def test_ramp_between_medium_and_dense(lj):
    # at 10 the input is half medium, half dense ((12 - 10) / 4, (10 - 8) / 4)
    assert abs(lj.ljsel_expert_suitability(_cfg(lj, "VL"), 10.0) - _good_clipped_at_half()) < TOL
    # cluster lists okay / okay there: okay clipped at 0.5, symmetric -> 0.5
    assert abs(lj.ljsel_expert_suitability(_cfg(lj, "CL"), 10.0) - 0.5) < TOL
    # window lists bad / bad: bad clipped at 0.5
    assert abs(lj.ljsel_expert_suitability(_cfg(lj, "VLW"), 10.0) - (1.0 - _good_clipped_at_half())) < TOL


def test_threshold_decisions(lj):
    # a dense liquid trials Verlet and cluster lists (0.5), not linked cells
    # or window lists; a dilute gas trials Verlet lists only
    r = {m: lj.ljsel_expert_suitability(_cfg(lj, m), 19.1) for m in ("VL", "VLW", "LC", "CL")}
    assert r["VL"] >= 0.5 and r["CL"] >= 0.5 - 1e-9 and r["LC"] < 0.5 and r["VLW"] < 0.5
    g = {m: lj.ljsel_expert_suitability(_cfg(lj, m), 0.3) for m in ("VL", "VLW", "LC", "CL")}
    assert g["VL"] >= 0.5 and g["LC"] < 0.5 and g["VLW"] < 0.5 and g["CL"] < 0.5


def test_invalid_arguments(lj):
    with pytest.raises(lj.LjselError):
        lj.ljsel_expert_suitability(_cfg(lj, "VL"), float("nan"))
