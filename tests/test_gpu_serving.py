"""Residency (streamed chunk blocks under an HBM budget) and the request loop.

* A streamed scene renders bit-identically to the same scene held resident
  (same keys, same pixels): the blocks only change where attributes are read.
* A budget that holds about two blocks forces eviction and reload along a
  trajectory; images are still identical.
* Requests served concurrently (continuous batching over slots) give the same
  image as the same request rendered alone.
* Failures are made on the host: an injected upload failure fails only the
  request that needed it; a budget no block fits fails requests cleanly.
"""
import numpy as np
import pytest

from paper_2505_23158_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_23158_gb300 import build
    build.build()
    from paper_2505_23158_gb300 import api
    return torch, api


@pytest.fixture(scope="module")
def scene_cams():
    scene, cams = synth.workload_outdoor(seed=2, n_poses=24, scale=0.04, width=320, height_px=180)
    return scene, cams


def _render(ctx, sid, mode, cam):
    out = np.empty((cam.height, cam.width, 3), np.float32)
    st = ctx.render_host(sid, mode, [cam], out)
    return out, st[0]


def test_streamed_equals_resident(env, scene_cams):
    torch, api = env
    scene, cams = scene_cams
    with api.Lodge(0) as ctx:
        r = ctx.load_scene(scene, api.RESIDENT)
        s = ctx.load_scene(scene, api.STREAMED)
        for mode in (api.CHUNK, api.CHUNK_BLEND):
            for cam in cams[::5]:
                a, sa = _render(ctx, r, mode, cam)
                b, sb = _render(ctx, s, mode, cam)
                assert sa["n_active"] == sb["n_active"] and sa["n_keys"] == sb["n_keys"]
                assert np.array_equal(a, b)
            # key lists and selected gids are identical too
            img, st, h = ctx.render(s, mode, cams[3], save=True)
            k1, g1 = ctx.debug_keys(h)
            ctx.release(h)
            img, st, h = ctx.render(r, mode, cams[3], save=True)
            k2, g2 = ctx.debug_keys(h)
            ctx.release(h)
            assert torch.equal(k1, k2) and torch.equal(g1, g2)
            sel_s, gs = ctx.select(s, mode, cams[3], want_gids=True)
            sel_r, gr = ctx.select(r, mode, cams[3], want_gids=True)
            assert sel_s == sel_r and torch.equal(gs, gr)
        with pytest.raises(api.LodgeError) as e:
            _render(ctx, s, api.FULL, cams[0])
        assert e.value.status == 4
        st = ctx.residency_stats()
        assert st["block_uploads"] > 0 and st["block_hits"] > 0


def test_eviction_under_tight_budget(env, scene_cams):
    torch, api = env
    scene, cams = scene_cams
    # measure the scratch a frame needs and the size of a block without a
    # budget, then allow scratch plus about 2.5 blocks (the scene has 9)
    with api.Lodge(0) as probe:
        s = probe.load_scene(scene, api.STREAMED)
        ws_max, blk = 0.0, 0.0
        for cam in cams:
            _render(probe, s, api.CHUNK_BLEND, cam)
            st = probe.residency_stats()
            blk = st["upload_bytes"] / max(st["block_uploads"], 1) * 1.1
            ws_max = max(ws_max, st["hbm_used"] - st["resident_blocks"] * blk)
        assert st["resident_blocks"] >= 4
        budget = int(ws_max + 2.5 * blk * 1.2)
    with api.Lodge(0) as ref, api.Lodge(0, hbm_budget_bytes=budget) as ctx:
        r = ref.load_scene(scene, api.RESIDENT)
        s = ctx.load_scene(scene, api.STREAMED)
        for cam in cams:
            a, _ = _render(ref, r, api.CHUNK_BLEND, cam)
            b, _ = _render(ctx, s, api.CHUNK_BLEND, cam)
            assert np.array_equal(a, b)
        st = ctx.residency_stats()
        assert st["block_evictions"] > 0, st
        assert st["hbm_used"] <= budget


def test_serve_mix_equals_alone(env, scene_cams):
    torch, api = env
    scene, cams = scene_cams
    plain, pcams = synth.workload_plain(0)
    res_opts = [(320, 180), (160, 90), (256, 144), (96, 64)]
    with api.Lodge(0) as ctx:
        s = ctx.load_scene(scene, api.STREAMED)
        p = ctx.load_scene(plain, api.RESIDENT)
        reqs = []
        for i in range(32):
            w, h = res_opts[i % 4]
            if i % 3 == 2:
                cam = synth.plain_camera(w, h)
                reqs.append((p, api.FULL, cam, 0.002 * i))
            else:
                c = cams[(7 * i) % len(cams)]
                cam = synth.look_at(c.center, c.R[2].astype(np.float64), (0, 0, 1), w, h, 70.0)
                reqs.append((s, api.CHUNK_BLEND if i % 2 else api.CHUNK, cam, 0.002 * i))
        results, imgs = ctx.serve(reqs, slots=4, realtime=True, images=True)
        assert all(r["status"] == 0 for r in results), [r["status"] for r in results]
        assert len({r["slot"] for r in results}) > 1        # requests ran on several slots
        for (sid, mode, cam, _), img in zip(reqs, imgs):
            alone, _ = _render(ctx, sid, mode, cam)
            assert np.array_equal(alone, img)
        lat = np.array([r["latency_s"] for r in results])
        assert np.all(lat > 0)


def test_injected_upload_failure_fails_one_request(env, scene_cams):
    torch, api = env
    scene, cams = scene_cams
    with api.Lodge(0) as ctx:
        s = ctx.load_scene(scene, api.STREAMED)
        ctx.inject_upload_failures(1)
        reqs = [(s, api.CHUNK_BLEND, cams[i], 0.0) for i in range(6)]
        results, imgs = ctx.serve(reqs, slots=1, realtime=False, images=True)
        status = [r["status"] for r in results]
        assert status.count(3) == 1 and status.count(0) == 5, status
        for (sid, mode, cam, _), img, r in zip(reqs, imgs, results):
            if r["status"] == 0:
                alone, _ = _render(ctx, sid, mode, cam)
                assert np.array_equal(alone, img)
        assert ctx.residency_stats()["failed_uploads"] == 1


def test_budget_too_small_fails_cleanly(env, scene_cams):
    torch, api = env
    scene, cams = scene_cams
    with api.Lodge(0) as probe:
        s = probe.load_scene(scene, api.STREAMED)
        base = probe.residency_stats()["hbm_used"]
    # room for loading (a temporary device copy of the means) but for no chunk block
    budget = base + 12 * scene.n_total + (8 << 20)
    with api.Lodge(0, hbm_budget_bytes=budget) as ctx:
        s = ctx.load_scene(scene, api.STREAMED)
        results, _ = ctx.serve([(s, api.CHUNK_BLEND, cams[0], 0.0)], slots=1, realtime=False,
                               wait_limit_s=0.2)
        assert results[0]["status"] == 6
        # the context is still usable
        assert ctx.residency_stats()["hbm_used"] <= budget


def test_batch_render_equals_single(env, scene_cams):
    """One compositing launch for frames of different scenes, modes and sizes
    gives the images of rendering each frame alone, bit for bit."""
    torch, api = env
    scene, cams = scene_cams
    plain, pcams = synth.workload_plain(0)
    with api.Lodge(0) as ctx:
        r = ctx.load_scene(scene, api.RESIDENT)
        s = ctx.load_scene(scene, api.STREAMED)
        p = ctx.load_scene(plain, api.RESIDENT)
        frames = []
        for i in range(12):
            c = cams[(5 * i) % len(cams)]
            w, h = [(320, 180), (160, 90), (256, 144)][i % 3]
            cam = synth.look_at(c.center, c.R[2].astype(np.float64), (0, 0, 1), w, h, 70.0)
            sid, mode = [(r, api.CHUNK_BLEND), (s, api.CHUNK), (r, api.LOD), (s, api.CHUNK_BLEND)][i % 4]
            frames.append((sid, mode, cam))
        frames.append((p, api.FULL, pcams[0]))
        # the first batch sizes each slot's key capacity (mid-frame syncs);
        # the second runs every resident frame without its mid-frame sync
        for rep in range(2):
            imgs, stats = ctx.render_batch(frames)
            for (sid, mode, cam), img, st in zip(frames, imgs, stats):
                alone, st1 = ctx.render(sid, mode, cam)
                assert torch.equal(alone, img), rep
                assert st1["n_keys"] == st["n_keys"] and st1["n_visible"] == st["n_visible"]


def test_batch_frames_outgrowing_capacity_rendered_again(env):
    """A batch whose slots were sized by frames that saw nothing: the next
    batch's frames outgrow the key capacity, are rendered again alone, and
    every image and count equals the camera rendered alone."""
    torch, api = env
    scene, cams = synth.workload_outdoor(seed=8, n_poses=12, scale=0.02, width=320, height_px=180)
    up = np.asarray(cams[0].center, np.float64)
    away = synth.look_at(up + np.array([0.0, 0.0, 1000.0]), up + np.array([0.0, 0.0, 2000.0]), (1, 0, 0),
                         320, 180, 70.0)
    with api.Lodge(0) as ctx:
        sid = ctx.load_scene(scene)
        ctx.set_bin_size(1)
        ctx.render_batch([(sid, api.FULL, away)] * 4)
        ctx.profile_enable(True)
        frames = [(sid, api.FULL, c) for c in cams[:4]]
        imgs, stats = ctx.render_batch(frames)
        prof = ctx.profile_read()
        ctx.profile_enable(False)
        assert prof["redone"] >= 1, prof
        for (_, mode, cam), img, st in zip(frames, imgs, stats):
            one, st1 = ctx.render(sid, mode, cam)
            assert torch.equal(one, img)
            assert st1["n_keys"] == st["n_keys"] and st1["n_visible"] == st["n_visible"]


def test_serve_batched_steps_equal_alone(env, scene_cams):
    """The serving loop in step mode (each step's frames composited by one
    launch): every image equals the same request rendered alone."""
    torch, api = env
    scene, cams = scene_cams
    with api.Lodge(0) as ctx:
        s = ctx.load_scene(scene, api.STREAMED)
        reqs = []
        for i in range(24):
            w, h = [(320, 180), (160, 90), (96, 64)][i % 3]
            c = cams[(7 * i) % len(cams)]
            cam = synth.look_at(c.center, c.R[2].astype(np.float64), (0, 0, 1), w, h, 70.0)
            reqs.append((s, api.CHUNK_BLEND if i % 2 else api.CHUNK, cam, 0.001 * i))
        # all requests are there at once (not realtime): steps of 8 frames
        results, imgs = ctx.serve(reqs, realtime=False, images=True, batch=8)
        assert all(r["status"] == 0 for r in results), [r["status"] for r in results]
        assert max(r["slot"] for r in results) == 7          # full steps of 8 frames
        assert all(r["step_frames"] == 8 for r in results)
        for (sid, mode, cam, _), img in zip(reqs, imgs):
            alone, _ = _render(ctx, sid, mode, cam)
            assert np.array_equal(alone, img)
