"""Greedy depth-threshold search (Sec. 3, "Selecting depth thresholds") on
the GPU (one K10 pass per view and step, all candidates at once) against
the oracle's plain search (one LOD selection and key count per candidate):
chosen thresholds and every candidate's key total bit-exact."""
import numpy as np
import pytest

import oracle as O
from paper_2505_23158_gb300 import synth

pytestmark = pytest.mark.gpu

L0 = [k + 0.5 for k in range(1, 31)]
L1 = [b + f for b in (0.0, 2.0, 4.0, 6.0, 8.0) for f in (1.0, 1.3, 1.7)] + [11.0 + 2 * k for k in range(15)]
L2 = [b + f for b in (12.0, 14.0, 16.0, 18.0) for f in (0.2, 0.5, 0.8)]


@pytest.fixture(scope="module")
def api():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_23158_gb300 import build
    build.build()
    from paper_2505_23158_gb300 import api
    return api


def test_ray_scene_matches_oracle(api):
    scene, cam = synth.ray_scene([L0, L1, L2])
    cand = sorted([2.0 * k for k in range(1, 21)] + [10.4])
    d_ref, t_ref = O.select_thresholds(O.OracleScene(scene), [cam], cand)
    with api.Lodge(0) as ctx:
        sid = ctx.load_scene(scene)
        d, t = ctx.select_thresholds(sid, [cam], cand)
    assert list(d) == [10.0, 20.0] == d_ref
    assert np.array_equal(t, t_ref)


@pytest.mark.parametrize("residency", ["RESIDENT", "STREAMED"])
def test_outdoor_matches_oracle(api, residency):
    scene, cams = synth.workload_outdoor(seed=3, n_poses=40, scale=0.02, width=640, height_px=360)
    views = cams[::10]
    cand = [2.5 * 1.25 ** k for k in range(20)]
    d_ref, t_ref = O.select_thresholds(O.OracleScene(scene), views, cand)
    with api.Lodge(0) as ctx:
        sid = ctx.load_scene(scene, getattr(api, residency))
        d, t = ctx.select_thresholds(sid, views, cand)
    assert np.array_equal(t, t_ref)
    assert list(d) == list(d_ref)
    assert (t[0] > 0).sum() == len(cand)


def test_bad_candidates_rejected(api):
    scene, cam = synth.ray_scene([L0, L1])
    with api.Lodge(0) as ctx:
        sid = ctx.load_scene(scene)
        for bad in ([5.0, 5.0], [5.0, 3.0], [-1.0], [float("inf")]):
            with pytest.raises(api.LodgeError) as e:
                ctx.select_thresholds(sid, [cam], bad)
            assert e.value.status == 1
