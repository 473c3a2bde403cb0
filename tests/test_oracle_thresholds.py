"""Pins of the oracle's greedy depth-threshold search (Sec. 3, "Selecting
depth thresholds").

On ``synth.ray_scene`` every Gaussian yields exactly one tile key, so the
cost of a threshold set (keys summed over the views) is a count of
Gaussians by distance band (Eq. 2) that needs no projection: these tests
recount it from the distances alone and check the searched thresholds
against the optimum worked out by hand in the comments.
"""
import math

import numpy as np

import oracle as O
from paper_2505_23158_gb300 import synth

# level 0: one Gaussian per metre, at 1.5, 2.5, ..., 30.5 m
L0 = [k + 0.5 for k in range(1, 31)]
# level 1: three per 2 m interval below 10 m, one per 2 m interval beyond
L1 = [b + f for b in (0.0, 2.0, 4.0, 6.0, 8.0) for f in (1.0, 1.3, 1.7)] + [11.0 + 2 * k for k in range(15)]
# level 2: three per 2 m interval in [12, 20) m, none beyond
L2 = [b + f for b in (12.0, 14.0, 16.0, 18.0) for f in (0.2, 0.5, 0.8)]
CANDIDATES = [2.0 * k for k in range(1, 21)] + [10.4]
CANDIDATES = sorted(CANDIDATES)


def count_cost(d):
    """Keys of LOD rendering with inner thresholds d on the ray scene: the
    number of Gaussians inside their level's band [d_l, d_{l+1})."""
    bands = [0.0] + list(d) + [math.inf]
    n = 0
    for l, dl in enumerate((L0, L1, L2)[:len(bands) - 1]):
        n += sum(1 for x in dl if bands[l] <= x < bands[l + 1])
    return n


def test_greedy_thresholds_on_ray_scene():
    scene, cam = synth.ray_scene([L0, L1, L2])
    osc = O.OracleScene(scene)
    d, table = O.select_thresholds(osc, [cam], CANDIDATES)
    # step 1 (levels 0 and 1): cost(x = 2k) = (2k - 1) + (30 - 3k) = 29 - k
    # for k <= 5 and (2k - 1) + (20 - k) = 19 + k above, so 24 at x = 10,
    # tied by x = 10.4 (no Gaussian lies in [10, 10.4)): the smaller wins.
    assert d[0] == 10.0
    # step 2 (d_1 = 10): cost(x = 2k) = 9 + (k - 5) + 3 (10 - k) = 34 - 2k up
    # to x = 20 and 9 + (k - 5) beyond: 14 at x = 20; x = 10.4 gives 21.
    assert d[1] == 20.0
    for k, x in enumerate(CANDIDATES):
        assert table[0, k] == count_cost([x, math.inf]), x
        if x > 10.0:
            assert table[1, k] == count_cost([10.0, x]), x
        else:
            assert table[1, k] == -1
    assert table[0, CANDIDATES.index(10.0)] == 24 == table[0, CANDIDATES.index(10.4)]
    assert table[1, CANDIDATES.index(20.0)] == 14


def test_views_add_and_candidates_run_out():
    scene, cam = synth.ray_scene([L0, L1, L2])
    osc = O.OracleScene(scene)
    # the same view twice doubles every cost and keeps the choice
    d1, t1 = O.select_thresholds(osc, [cam], CANDIDATES)
    d2, t2 = O.select_thresholds(osc, [cam, cam], CANDIDATES)
    assert d1 == d2
    assert np.array_equal(np.where(t1 >= 0, 2 * t1, -1), t2)
    # a single candidate: level 1 takes it, nothing is left for level 2
    d, t = O.select_thresholds(osc, [cam], [6.0])
    assert d[0] == 6.0 and math.isinf(d[1])
    assert t[0, 0] == count_cost([6.0, math.inf]) and t[1, 0] == -1


def test_single_level_has_no_thresholds():
    scene, cam = synth.ray_scene([L0])
    d, t = O.select_thresholds(O.OracleScene(scene), [cam], CANDIDATES)
    assert d == [] and t.shape == (0, len(CANDIDATES))
