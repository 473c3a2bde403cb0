"""Importance score and per-chunk visibility filtering (Sec. 3, "Importance
pruning" and "Visibility filtering", after RadSplat) on the GPU (K12: the
blend's walk recording each record's largest weight) against the oracle.

Scores: FP32 against FP64, so each GPU score must lie within 2e-4 of the
oracle's range [clean, all], where `clean` ignores pixels with a knife-edge
decision (alpha near 1/255, T near 1e-4) and `all` takes every pixel.
Filtering: the kept set equals the oracle's, except for Gaussians whose
score lies within that margin of the threshold."""
import numpy as np
import pytest

import oracle as O
from paper_2505_23158_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 2e-4


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_23158_gb300 import build
    build.build()
    from paper_2505_23158_gb300 import api
    return torch, api


def _check_scores(gpu, ref_all, ref_clean):
    lo = np.minimum(ref_clean, ref_all) - TOL
    hi = ref_all + TOL
    bad = np.flatnonzero((gpu < lo) | (gpu > hi))
    assert bad.size == 0, (bad[:5], gpu[bad[:5]], ref_clean[bad[:5]], ref_all[bad[:5]])


def test_plain_scene_scores(env):
    torch, api = env
    scene, cams = synth.workload_plain(0)
    osc = O.OracleScene(scene)
    g = np.arange(scene.n_total)
    ref, clean = O.importance(osc, cams[0], g)
    with api.Lodge(0) as ctx:
        sid = ctx.load_scene(scene)
        sc = ctx.importance(sid, api.FULL, cams).cpu().numpy().astype(np.float64)
    _check_scores(sc, ref, clean)
    assert (sc > 0).sum() > 1000


def test_outdoor_blend_scores_over_views(env):
    torch, api = env
    scene, cams = synth.workload_outdoor(seed=4, n_poses=40, scale=0.02, width=320, height_px=180)
    osc = O.OracleScene(scene)
    views = cams[::8]
    ref = np.zeros(scene.n_total)
    clean = np.zeros(scene.n_total)
    for cam in views:
        g, m, _ = O.active_set(osc, O.MODE_CHUNK_BLEND, cam)
        a, c = O.importance(osc, cam, g, m)
        ref[g] = np.maximum(ref[g], a)
        clean[g] = np.maximum(clean[g], c)
    with api.Lodge(0) as ctx:
        for res in (api.RESIDENT, api.STREAMED):
            sid = ctx.load_scene(scene, res)
            sc = ctx.importance(sid, api.CHUNK_BLEND, views).cpu().numpy().astype(np.float64)
            _check_scores(sc, ref, clean)


def test_chunk_visibility_filtering(env):
    torch, api = env
    scene, cams = synth.workload_outdoor(seed=5, n_poses=10, scale=0.02, width=320, height_px=180)
    osc = O.OracleScene(scene)
    K = scene.chunk_centers.shape[0]
    chunk = K // 2
    views = synth.chunk_views(scene, chunk, seed=1, n=6, width=320, height_px=180)
    members = O.chunk_select(osc, chunk)
    ref = np.zeros(members.size)
    clean = np.zeros(members.size)
    for cam in views:
        a, c = O.importance(osc, cam, members)
        ref = np.maximum(ref, a)
        clean = np.maximum(clean, c)
    thr = 0.02
    with api.Lodge(0) as ctx:
        sid = ctx.load_scene(scene)
        score = ctx.importance(sid, api.CHUNK, views, chunk=chunk)
        sc = score.cpu().numpy().astype(np.float64)
        _check_scores(sc[members], ref, clean)
        n_kept = ctx.filter_chunk(sid, chunk, score, thr)
        cam = views[0]
        sel, gids = ctx.select(sid, api.CHUNK, cam, want_gids=True)
        assert sel["chunk_a"] == chunk and sel["n_active"] == n_kept
        kept = (gids.cpu().numpy().view(np.uint32) & 0x3FFFFFFF).astype(np.int64)
    sure = (np.abs(ref - thr) > TOL) & (np.abs(clean - thr) > TOL)
    want = set(members[(ref >= thr) & sure].tolist())
    unsure = set(members[~sure].tolist())
    got = set(kept.tolist())
    assert want <= got and got - want <= unsure
    assert np.all(np.diff(kept) > 0)
    assert 0 < n_kept < members.size
