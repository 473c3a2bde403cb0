"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars (fixed here, derived in the design notes):
  * selected sets, chunk choices, culling, tile rects, sorted tile keys:
    bit-exact;
  * pixels: on clamp(rgb, 0, 1), max-abs <= 2e-4 per channel and mean-abs
    <= 1e-5 over all pixels.  Where the FP32 error bound of a decision of
    Eq. 1 (the 1/255 skip, the T < 1e-4 stop) spans its threshold (a knife
    edge), either way is a correct render: such a pixel is compared with
    the range of the oracle's results over those choices, not left out.
    Pixels whose choices the oracle cannot enumerate may be at most 1e-5 of
    the image.  Each comparison prints its knife-edge counts.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2505_23158_gb300 import synth

pytestmark = pytest.mark.gpu

MAX_ABS = 2e-4
MEAN_ABS = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    from paper_2505_23158_gb300 import build
    build.build()
    from paper_2505_23158_gb300.api import Lodge
    c = Lodge(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def plain_loaded(ctx):
    scene, cams = synth.workload_plain(0)
    return scene, cams, O.OracleScene(scene), ctx.load_scene(scene)


def compare_images(gpu, ref, tag=""):
    try:
        out = O.compare_pixels(gpu, ref, max_abs=MAX_ABS, mean_abs=MEAN_ABS)
    except AssertionError as e:
        raise AssertionError(f"{tag}: {e}") from None
    print(f"[pixels] {tag}: {out}")
    return out


def oracle_keys_u64(osc, cam, gids, mults=None):
    k, g = O.keys(osc, cam, gids, mults)
    return k, g


# ---------------------------------------------------------------------------
# plain single-level scene, FULL mode
# ---------------------------------------------------------------------------
def test_plain_keys_bit_exact(ctx, plain_loaded):
    from paper_2505_23158_gb300.api import FULL
    scene, cams, osc, sid = plain_loaded
    img, st, h = ctx.render(sid, FULL, cams[0], save=True)
    try:
        keys, gids = ctx.debug_keys(h)
        k_ref, g_ref = oracle_keys_u64(osc, cams[0], np.arange(osc.n_total))
        assert st["n_keys"] == k_ref.size
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), k_ref)
        assert np.array_equal(gids.cpu().numpy().astype(np.int64), g_ref)
    finally:
        ctx.release(h)


def test_plain_records(ctx, plain_loaded):
    from paper_2505_23158_gb300.api import FULL
    scene, cams, osc, sid = plain_loaded
    _, st, h = ctx.render(sid, FULL, cams[0], save=True)
    try:
        r = {k: v.cpu().numpy() for k, v in ctx.debug_records(h).items()}
    finally:
        ctx.release(h)
    pr = O.project(osc, cams[0], np.arange(osc.n_total))
    vis = np.flatnonzero(pr["visible"])
    assert np.array_equal(r["gid"].astype(np.int64), vis)
    assert np.array_equal(r["depth"].view(np.uint32), pr["z"][vis].view(np.uint32))
    assert np.array_equal(r["rect"], pr["rect"][vis])
    err2 = np.abs(r["mean2"] - pr["mean2"][vis]).max()
    print(f"[records] projected mean max error {err2:.3g} px")
    assert err2 < 1e-4
    assert np.abs(r["opacity"] - pr["opacity"][vis]).max() < 1e-6
    assert np.abs(r["rgb"] - pr["rgb"][vis]).max() < 2e-5
    rel = np.abs(r["conic"] - pr["conic"][vis]) / (np.abs(pr["conic"][vis]).max(axis=1, keepdims=True))
    assert rel.max() < 1e-4


def test_plain_image(ctx, plain_loaded):
    from paper_2505_23158_gb300.api import FULL
    scene, cams, osc, sid = plain_loaded
    img, st = ctx.render(sid, FULL, cams[0])
    ref = O.render(osc, cams[0], np.arange(osc.n_total))
    compare_images(img.cpu().numpy(), ref, "plain")
    assert st["n_visible"] == ref["n_visible"] and st["n_keys"] == ref["n_keys"]


@pytest.mark.parametrize("wh", [(100, 70), (17, 33), (1, 1), (16, 16), (257, 129)])
def test_ragged_image_sizes(ctx, plain_loaded, wh):
    from paper_2505_23158_gb300.api import FULL
    scene, cams, osc, sid = plain_loaded
    cam = synth.plain_camera(*wh)
    img, st, h = ctx.render(sid, FULL, cam, save=True)
    try:
        keys, gids = ctx.debug_keys(h)
    finally:
        ctx.release(h)
    k_ref, g_ref = oracle_keys_u64(osc, cam, np.arange(osc.n_total))
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), k_ref)
    ref = O.render(osc, cam, np.arange(osc.n_total))
    compare_images(img.cpu().numpy(), ref, f"{wh}")


def test_nothing_visible(ctx, plain_loaded):
    from paper_2505_23158_gb300.api import FULL
    scene, cams, osc, sid = plain_loaded
    cam = synth.look_at((0, 0, -3.0), (0, 0, -1.0), (0, -1, 0), 64, 48, 60.0)  # facing away
    img, st = ctx.render(sid, FULL, cam)
    assert st["n_visible"] == 0 and st["n_keys"] == 0
    assert float(img.abs().max()) == 0.0


def test_render_host_matches_device(ctx, plain_loaded):
    from paper_2505_23158_gb300.api import FULL
    scene, cams, osc, sid = plain_loaded
    img, _ = ctx.render(sid, FULL, cams[0])
    out = np.empty((cams[0].height, cams[0].width, 3), np.float32)
    ctx.render_host(sid, FULL, [cams[0]], out)
    assert np.array_equal(out, img.cpu().numpy())


def test_render_host_pinned_several_cameras(ctx, torch_cuda):
    """Host-buffer calls over several cameras into page-locked and pageable
    memory (each image copied back on its frame's stream as soon as it is
    done): each image equals the device render, for images of several sizes."""
    from paper_2505_23158_gb300.api import CHUNK_BLEND
    scene, cams = synth.workload_outdoor(seed=3, n_poses=8, scale=0.02, width=320, height_px=180)
    sid = ctx.load_scene(scene)
    sizes = [(320, 180), (17, 33), (64, 48), (33, 17), (320, 180)]
    cl = [synth.look_at(c.center, c.R[2].astype(np.float64), (0, 0, 1), w, h, 70.0)
          for c, (w, h) in zip(cams, sizes)]
    total = sum(c.width * c.height * 3 for c in cl)
    for pinned in (True, False):
        if pinned:
            host = torch_cuda.empty(total, dtype=torch_cuda.float32, pin_memory=True).numpy()
        else:
            host = np.empty(total, np.float32)
        host[:] = np.nan
        ctx.render_host(sid, CHUNK_BLEND, cl, host)
        off = 0
        for c in cl:
            k = c.width * c.height * 3
            one, _ = ctx.render(sid, CHUNK_BLEND, c)
            assert np.array_equal(host[off:off + k].reshape(c.height, c.width, 3), one.cpu().numpy()), (pinned, c.width)
            off += k


def test_repeatable(ctx, plain_loaded):
    from paper_2505_23158_gb300.api import FULL
    scene, cams, osc, sid = plain_loaded
    a, _ = ctx.render(sid, FULL, cams[0])
    a = a.clone()
    b, _ = ctx.render(sid, FULL, cams[0])
    assert bool((a == b).all())


# ---------------------------------------------------------------------------
# onesweep radix sort
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,bits", [(0, 32), (1, 32), (1000, 8), (3840, 32), (3841, 13),
                                    (100_000, 32), (1_000_003, 21), (2_000_000, 32)])
def test_sort_pairs_stable(ctx, torch_cuda, n, bits):
    torch = torch_cuda
    rng = np.random.default_rng(n + bits)
    hi = (1 << bits) if bits < 32 else (1 << 32)
    keys = rng.integers(0, hi, size=n, dtype=np.uint64).astype(np.uint32)
    if n > 10:
        keys[: n // 3] = keys[0]  # many equal keys: stability matters
        rng.shuffle(keys)
    vals = np.arange(n, dtype=np.uint32)
    kt = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    vt = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    ctx.sort_pairs(kt, vt, bits)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(kt.cpu().numpy().view(np.uint32), keys[order])
    assert np.array_equal(vt.cpu().numpy().view(np.uint32), vals[order])


def test_sort_pairs_partial_bits(ctx, torch_cuda):
    """Sorting on the low 13 bits leaves the order of keys that agree on them
    untouched (stable), whatever the high bits hold."""
    torch = torch_cuda
    rng = np.random.default_rng(1)
    keys = rng.integers(0, 1 << 32, size=50_000, dtype=np.uint64).astype(np.uint32)
    vals = np.arange(keys.size, dtype=np.uint32)
    kt = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    vt = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    ctx.sort_pairs(kt, vt, 13)
    order = np.argsort(keys & 0x1FFF, kind="stable")
    assert np.array_equal(vt.cpu().numpy().view(np.uint32), vals[order])


# ---------------------------------------------------------------------------
# outdoor LOD scene: selection, chunks, blending
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def outdoor(ctx):
    scene, cams = synth.workload_outdoor(seed=0, n_poses=6, scale=0.01, width=320, height_px=180)
    osc = O.OracleScene(scene)
    sid = ctx.load_scene(scene)
    return scene, cams, osc, sid


def _flags_from_oracle(osc, info):
    a = O.chunk_select(osc, info["A"])
    b = O.chunk_select(osc, info["B"])
    return a, b


@pytest.mark.parametrize("mode_name", ["LOD", "CHUNK", "CHUNK_BLEND"])
def test_outdoor_selection_bit_exact(ctx, outdoor, mode_name):
    from paper_2505_23158_gb300 import api
    mode = getattr(api, mode_name)
    scene, cams, osc, sid = outdoor
    for cam in cams:
        sel, gids = ctx.select(sid, mode, cam, want_gids=True)
        g_ref, m_ref, info = O.active_set(osc, mode, cam)
        raw = gids.cpu().numpy().view(np.uint32)
        assert np.array_equal((raw & 0x3FFFFFFF).astype(np.int64), g_ref)
        if mode_name == "LOD":
            assert sel["chunk_a"] == -1
            assert info["n_disagree"] <= 5
        else:
            assert sel["chunk_a"] == info["A"]
            if mode_name == "CHUNK_BLEND" and info["B"] >= 0:
                assert sel["chunk_b"] == info["B"]
                assert sel["t_a"] == info["tA"] and sel["t_b"] == info["tB"]
                a, b = _flags_from_oracle(osc, info)
                assert np.array_equal((raw >> 31) & 1, np.isin(g_ref, a).astype(np.uint32))
                assert np.array_equal((raw >> 30) & 1, np.isin(g_ref, b).astype(np.uint32))


@pytest.mark.parametrize("mode_name", ["FULL", "LOD", "CHUNK", "CHUNK_BLEND"])
def test_outdoor_render_parity(ctx, outdoor, mode_name):
    from paper_2505_23158_gb300 import api
    mode = getattr(api, mode_name)
    scene, cams, osc, sid = outdoor
    for i in (0, 3, 5):
        cam = cams[i]
        img, st, h = ctx.render(sid, mode, cam, save=True)
        try:
            keys, kg = ctx.debug_keys(h)
        finally:
            ctx.release(h)
        g_ref, m_ref, info = O.active_set(osc, mode, cam)
        k_ref, kg_ref = oracle_keys_u64(osc, cam, g_ref, m_ref)
        assert st["n_active"] == g_ref.size
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), k_ref), f"pose {i}"
        assert np.array_equal(kg.cpu().numpy().astype(np.int64), kg_ref)
        ref = O.render(osc, cam, g_ref, m_ref)
        compare_images(img.cpu().numpy(), ref, f"{mode_name} pose {i}")


def test_outdoor_multi_camera_batch(ctx, outdoor, torch_cuda):
    """Several cameras in one call equal one call per camera."""
    from paper_2505_23158_gb300.api import CHUNK_BLEND
    scene, cams, osc, sid = outdoor
    imgs, stats = ctx.render(sid, CHUNK_BLEND, cams[:3])
    for c, im in zip(cams[:3], imgs):
        one, _ = ctx.render(sid, CHUNK_BLEND, c)
        assert bool((one == im).all())


# ---------------------------------------------------------------------------
# errors
# ---------------------------------------------------------------------------
def test_invalid_arguments(ctx, plain_loaded):
    from paper_2505_23158_gb300.api import FULL, LodgeError
    scene, cams, osc, sid = plain_loaded
    with pytest.raises(LodgeError) as e:
        ctx.render(12345, FULL, cams[0])
    assert e.value.status == 1
    with pytest.raises(LodgeError):
        ctx.render(sid, 17, cams[0])
    bad = synth.plain_camera(0, 10)
    with pytest.raises(LodgeError):
        ctx.render(sid, FULL, bad)


def test_hbm_budget_enforced(torch_cuda):
    """A context whose budget cannot hold the scene refuses to load it
    (host-side failure, the device is untouched)."""
    from paper_2505_23158_gb300.api import Lodge, LodgeError
    scene, _ = synth.workload_plain(0)
    with Lodge(0, hbm_budget_bytes=64 * 1024) as c:
        with pytest.raises(LodgeError) as e:
            c.load_scene(scene)
        assert e.value.status == 6


def test_lod_with_randomised_thresholds(ctx, torch_cuda):
    """LOD renders whose thresholds are drawn per frame from U(0.7 d_l,
    1.3 d_l) (supplementary "LOD structure optimization steps"): selected
    counts, keys and pixels equal the oracle's for the same thresholds."""
    scene, cams = synth.workload_outdoor(seed=6, n_poses=20, scale=0.02, width=320, height_px=180)
    osc = O.OracleScene(scene)
    rng = np.random.default_rng(11)
    d0 = np.asarray(scene.d_thresholds, np.float64)
    views = cams[::5]
    d = np.stack([np.sort(d0 * rng.uniform(0.7, 1.3, size=d0.size)) for _ in views])
    sid = ctx.load_scene(scene)
    imgs, stats = ctx.render_lod(sid, views, d)
    for cam, dd, img, st in zip(views, d, imgs, stats):
        g, _ = O.lod_select(osc, cam.center, dd)
        ref = O.render(osc, cam, g)
        assert st["n_active"] == g.size and st["n_keys"] == ref["n_keys"]
        compare_images(img.cpu().numpy(), ref, "randomised LOD")


@pytest.mark.parametrize("which", ["plain", "outdoor"])
def test_compensated_2d_filter(ctx, torch_cuda, which):
    """Scenes rendered with Mip-Splatting's opacity-compensated 2D filter:
    keys bit-exact (the compensation enters the opacity cull and extent) and
    pixels within the bars."""
    from paper_2505_23158_gb300.api import CHUNK_BLEND, FULL
    if which == "plain":
        scene, cams = synth.workload_plain(0)
        mode, omode = FULL, O.MODE_FULL
    else:
        scene, cams = synth.workload_outdoor(seed=7, n_poses=10, scale=0.02, width=320, height_px=180)
        cams = cams[::3]
        mode, omode = CHUNK_BLEND, O.MODE_CHUNK_BLEND
    scene.filter2d = True
    osc = O.OracleScene(scene)
    sid = ctx.load_scene(scene)
    for cam in cams:
        g, m, _ = O.active_set(osc, omode, cam)
        img, st, h = ctx.render(sid, mode, cam, save=True)
        keys, _ = ctx.debug_keys(h)
        ctx.release(h)
        k_ref, _ = O.keys(osc, cam, g, m)
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), k_ref)
        ref = O.render(osc, cam, g, m)
        compare_images(img.cpu().numpy(), ref, f"filter2d {which}")


@pytest.mark.parametrize("log2", [3, 0])
def test_camera_list_equals_single_frames(ctx, torch_cuda, log2):
    """A render call over several cameras (its frames take turns on several
    streams, without mid-frame syncs for binned lists, and their compositing
    shares the SMs) gives each camera's single-frame image bit for bit, for
    every mode, with binned and per-tile key lists."""
    from paper_2505_23158_gb300.api import CHUNK, CHUNK_BLEND, FULL, LOD
    scene, cams = synth.workload_outdoor(seed=8, n_poses=12, scale=0.02, width=320, height_px=180)
    sid = ctx.load_scene(scene)
    try:
        ctx.set_bin_size(log2)
        for mode in (FULL, LOD, CHUNK, CHUNK_BLEND):
            imgs, stats = ctx.render(sid, mode, list(cams[:7]))
            for cam, img, st in zip(cams[:7], imgs, stats):
                one, st1 = ctx.render(sid, mode, cam)
                assert torch_cuda.equal(one, img)
                assert st1["n_keys"] == st["n_keys"]
    finally:
        ctx.set_bin_size(-1)


# ---------------------------------------------------------------------------
# key lists per bin of 2^k x 2^k tiles


def _bin_keys(rect, k):
    """Keys of one frame with bins of 2^k tiles square, from the oracle's
    tile rects (tx0, ty0, tx1, ty1): one per (record, bin) the rect touches."""
    r = rect.astype(np.int64) >> k
    return int(((r[:, 2] - r[:, 0] + 1) * (r[:, 3] - r[:, 1] + 1)).sum())


@pytest.mark.parametrize("log2", [0, 1, 2, 3])
def test_binned_lists_same_image(ctx, outdoor, torch_cuda, log2):
    """Compositing from per-bin lists gives the per-tile lists' image bit for
    bit and matches the oracle; the keys emitted and sorted are exactly one
    per (visible Gaussian, bin its tile rect touches)."""
    from paper_2505_23158_gb300.api import CHUNK_BLEND, FULL
    scene, cams, osc, sid = outdoor
    try:
        for mode in (FULL, CHUNK_BLEND):
            for i in (0, 4):
                cam = cams[i]
                ctx.set_bin_size(0)
                per_tile, st0 = ctx.render(sid, mode, cam)
                ctx.set_bin_size(log2)
                ctx.profile_enable(True)
                img, st = ctx.render(sid, mode, cam)
                prof = ctx.profile_read()
                ctx.profile_enable(False)
                assert torch_cuda.equal(img, per_tile), f"mode {mode} pose {i}"
                assert st["n_keys"] == st0["n_keys"]
                g_ref, m_ref, info = O.active_set(osc, mode, cam)
                pr = O.project(osc, cam, g_ref, m_ref)
                assert prof["frames"] == 1
                assert prof["keys"] == st["n_keys"]
                assert prof["bin_keys"] == _bin_keys(pr["rect"][pr["visible"]], log2)
                ref = O.render(osc, cam, g_ref, m_ref)
                compare_images(img.cpu().numpy(), ref, f"bins {log2} pose {i}")
    finally:
        ctx.set_bin_size(-1)


@pytest.mark.parametrize("wh", [(17, 33), (1, 1), (257, 129), (100, 70)])
def test_binned_lists_ragged_sizes(ctx, plain_loaded, torch_cuda, wh):
    """Bins that overhang the image edge (tiles_x, tiles_y not multiples of
    the bin size): same image as per-tile lists for every bin size."""
    from paper_2505_23158_gb300.api import FULL
    scene, cams, osc, sid = plain_loaded
    cam = synth.plain_camera(*wh)
    try:
        ctx.set_bin_size(0)
        ref, _ = ctx.render(sid, FULL, cam)
        for k in (1, 2, 3):
            ctx.set_bin_size(k)
            img, _ = ctx.render(sid, FULL, cam)
            assert torch_cuda.equal(img, ref), f"bins {k}"
    finally:
        ctx.set_bin_size(-1)


def test_bin_size_argument_checked(ctx):
    from paper_2505_23158_gb300.api import LodgeError
    for bad in (-2, 4):
        with pytest.raises(LodgeError):
            ctx.set_bin_size(bad)
    ctx.set_bin_size(-1)


@pytest.mark.parametrize("log2", [-1, 0, 1, 3])
def test_filtered_walk_equals_unfiltered(ctx, torch_cuda, log2):
    """The compositing walk that skips, per 8x8 pixel block, the records
    whose rect misses the block or whose ellipse reaches none of its pixel
    centres gives the image of the walk that visits every record of the
    tile's list (the one frames kept for the adjoint use), bit for bit: on
    the plain workload's anisotropic splats and on outdoor frames with near,
    large and off-axis splats."""
    dev = torch_cuda.device("cuda")
    cases = []
    scene, cams = synth.workload_plain(0)
    cases.append((scene.levels[0], cams[:2]))
    scene2, cams2 = synth.workload_outdoor(seed=3, n_poses=6, scale=0.01, width=320, height_px=180)
    cases.append((scene2.levels[0], cams2[:3]))
    try:
        ctx.set_bin_size(log2)
        for lv, cs in cases:
            n = lv.n
            ps = [torch_cuda.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev)
                  for a in (lv.means, lv.log_scales, lv.quats, lv.opacity_logits, lv.sh.reshape(n, 48))]
            for cam in cs:
                img, st, _ = ctx.render_params(*ps, cam, save=False)
                ref, st2, h = ctx.render_params(*ps, cam, save=True)
                ctx.release(h)
                assert st["n_keys"] == st2["n_keys"]
                assert torch_cuda.equal(img, ref)
    finally:
        ctx.set_bin_size(-1)


@pytest.mark.parametrize("log2", [0, 2])
def test_counting_mode_pairs(ctx, outdoor, torch_cuda, log2):
    """Counting mode: the compositing's composited (pixel, Gaussian) pairs
    equal the oracle's per-pixel contributor counts summed (up to knife-edge
    pixels), evaluations lie between that and the full per-tile walk, and
    the image is the plain kernel's."""
    from paper_2505_23158_gb300.api import CHUNK_BLEND
    scene, cams, osc, sid = outdoor
    cam = cams[2]
    try:
        ctx.set_bin_size(log2)
        plain, _ = ctx.render(sid, CHUNK_BLEND, cam)
        ctx.profile_enable(True, count_pairs=True)
        img, st = ctx.render(sid, CHUNK_BLEND, cam)
        prof = ctx.profile_read()
        ctx.profile_enable(False)
    finally:
        ctx.set_bin_size(-1)
    assert torch_cuda.equal(img, plain)
    g_ref, m_ref, info = O.active_set(osc, CHUNK_BLEND, cam)
    ref = O.render(osc, cam, g_ref, m_ref)
    used_ref = int(ref["ncontrib"].sum())
    assert used_ref > 0
    assert abs(prof["blend_pairs_used"] - used_ref) <= max(10, 1e-3 * used_ref), (prof, used_ref)
    assert prof["blend_pairs_used"] <= prof["blend_pairs"] <= ref["n_pairs_eval"]


def test_deferred_frames_overflow_rendered_again(torch_cuda):
    """A camera list whose first frames see nothing sizes its streams' key
    capacity small; the later frames outgrow it, are rendered again, and
    every image and count equals the camera rendered alone."""
    from paper_2505_23158_gb300 import api
    scene, cams = synth.workload_outdoor(seed=8, n_poses=12, scale=0.02, width=320, height_px=180)
    c0 = cams[0]
    up = np.asarray(c0.center, np.float64)
    away = synth.look_at(up + np.array([0.0, 0.0, 1000.0]), up + np.array([0.0, 0.0, 2000.0]), (1, 0, 0),
                         320, 180, 70.0)
    seq = [away, away] + list(cams[:6])
    with api.Lodge(0) as c2:
        sid = c2.load_scene(scene)
        c2.set_bin_size(1)
        c2.profile_enable(True)
        imgs, stats = c2.render(sid, api.FULL, seq)
        prof = c2.profile_read()
        c2.profile_enable(False)
        assert stats[0]["n_visible"] == 0 and stats[2]["n_keys"] > 0
        assert prof["redone"] >= 1, prof
        assert prof["frames"] == len(seq)
        for cam, img, st in zip(seq, imgs, stats):
            one, st1 = c2.render(sid, api.FULL, cam)
            assert torch_cuda.equal(one, img)
            assert st1["n_keys"] == st["n_keys"] and st1["n_visible"] == st["n_visible"]


def test_deferred_frames_with_nothing_visible(torch_cuda):
    """Frames that see nothing in the middle of a camera list (their counts
    stay on the device: every sort and the emission run with a count of 0)
    render black and leave the following frames unchanged."""
    from paper_2505_23158_gb300 import api
    scene, cams = synth.workload_outdoor(seed=5, n_poses=12, scale=0.02, width=320, height_px=180)
    up = np.asarray(cams[0].center, np.float64)
    away = synth.look_at(up + np.array([0.0, 0.0, 1000.0]), up + np.array([0.0, 0.0, 2000.0]), (1, 0, 0),
                         320, 180, 70.0)
    seq = list(cams[:4]) + [away] * 4 + list(cams[4:8])
    with api.Lodge(0) as c2:
        sid = c2.load_scene(scene)
        for mode in (api.CHUNK_BLEND, api.FULL):
            imgs, stats = c2.render(sid, mode, seq)
            for k in range(4, 8):
                assert stats[k]["n_visible"] == 0 and stats[k]["n_keys"] == 0
                assert float(imgs[k].abs().max()) == 0.0
            for cam, img, st in zip(seq, imgs, stats):
                one, st1 = c2.render(sid, mode, cam)
                assert torch_cuda.equal(one, img)
                assert st1["n_keys"] == st["n_keys"]


def _dense_cluster_scene(n, seed=5):
    """n small, nearly opaque Gaussians packed into a 5 cm cube that the
    256x256 plain camera sees inside one 16x16 tile (pixels 144..159 in x and
    y): that tile's bin holds every one of them."""
    rng = np.random.default_rng(seed)
    lvl = synth.Level((rng.uniform(-0.025, 0.025, (n, 3)) + [0.325, 0.325, 0.0]).astype(np.float32),
                      np.full((n, 3), np.log(0.004), np.float32),
                      rng.normal(size=(n, 4)).astype(np.float32),
                      np.full(n, 2.0, np.float32),
                      rng.normal(0, 0.3, (n, 16, 3)).astype(np.float32))
    return synth.Scene(levels=[lvl], d_thresholds=np.zeros(0), chunk_centers=np.zeros((1, 3)))


@pytest.mark.parametrize("log2", [1, 3])
def test_deferred_frames_equal_synced_frames_dense_bins(ctx, torch_cuda, log2):
    """Frames of a camera list that run without a mid-frame sync (capacities,
    counts on the device) give the images of frames with their sync (here in
    counting mode) bit for bit, also when one bin holds thousands of keys: on
    the plain workload (bins of hundreds to about 1300 keys) and on clusters
    of 6000 and 30000 Gaussians inside one tile."""
    from paper_2505_23158_gb300.api import FULL
    scene, cams = synth.workload_plain(0)
    cam = synth.plain_camera(256, 256)
    cases = [(ctx.load_scene(scene), cams[:3]),
             (ctx.load_scene(_dense_cluster_scene(6000)), [cam] * 3),
             (ctx.load_scene(_dense_cluster_scene(30000)), [cam] * 3)]
    try:
        ctx.set_bin_size(log2)
        for sid, cs in cases:
            ctx.profile_enable(True, count_pairs=True)
            refs = [ctx.render(sid, FULL, c)[0].clone() for c in cs]
            ctx.profile_enable(False)
            ctx.render(sid, FULL, cs[0])           # the slot learns its key capacity
            imgs, _ = ctx.render(sid, FULL, list(cs))
            for img, ref in zip(imgs, refs):
                assert torch_cuda.equal(img, ref)
    finally:
        ctx.set_bin_size(-1)


def test_long_camera_list_stats_and_images(ctx, plain_loaded, torch_cuda):
    """A call over 300 cameras: each of the eight render slots gets more
    frames than its 32-entry status ring holds, so the ring is taken entry by
    entry while later frames run; every frame's stats equal the camera
    rendered alone, and a sample of images equals the single renders bit for
    bit."""
    from paper_2505_23158_gb300.api import FULL
    scene, cams, osc, sid = plain_loaded
    rng = np.random.default_rng(9)
    cl = []
    for i in range(300):
        eye = (rng.uniform(-0.4, 0.4), rng.uniform(-0.4, 0.4), -3.0 + rng.uniform(-0.3, 0.3))
        cl.append(synth.look_at(eye, (0.0, 0.0, 1.0), (0, -1, 0), 64, 48, 60.0))
    imgs, stats = ctx.render(sid, FULL, cl)
    for i in list(range(0, 300, 7)) + [299]:
        one, st = ctx.render(sid, FULL, cl[i])
        assert st["n_keys"] == stats[i]["n_keys"] and st["n_visible"] == stats[i]["n_visible"], i
        if i % 21 == 0 or i == 299:
            assert torch_cuda.equal(one, imgs[i]), i
