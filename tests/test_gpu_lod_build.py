"""The per-level LOD build (supplementary "LOD structure optimization
steps") on the GPU path, against the oracle's importance score.

Level 1 of the fine-tuning scene (one 62.5 m chunk cell of the outdoor
generator) is built from its level 0 with d_1 = 10 m: the copy gets the
Eq. 3 filter of depth d_1, then three rounds prune at 0.2, 0.6 and 1.0 of
gamma by importance over LOD renders of the views and run 1000 steps with
d_1 drawn from U(7, 13) m, updating level 1 only.  The target images are the
full-detail renders of level 0 (the representation the LOD level stands in
for).  Checks:
  * the importance scores the GPU prunes by lie within the oracle's
    knife-edge bracket [clean - 2e-4, all + 2e-4] for every Gaussian of the
    trained level, in every round, and the kept set equals the oracle's
    except for Gaussians whose score is within that margin of the threshold;
  * the fine-tuning steps of every round lower the objective they sample
    (0.8 L1 + 0.2 (1 - SSIM), the mean over the views and over d_1 at 0.7,
    0.85, 1.0, 1.15 and 1.3 of 10 m) below its value after the pruning;
  * level 0 is never changed.
"""
import numpy as np
import pytest

import oracle as O
from paper_2505_23158_gb300 import synth

pytestmark = pytest.mark.gpu

MARGIN = 2e-4


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_23158_gb300 import api, build
    build.build()
    return torch, api


def _oracle_scores(lv0, params, fv, d1, views):
    """Per-Gaussian importance of the trained level in the oracle: LOD
    frames over [level 0, trained level] at threshold d1; returns the
    (all, clean) maxima over the views."""
    m, ls, q, lg, sh = params
    n = m.shape[0]
    lvl = synth.Level(m, ls, q, lg, np.asarray(sh, np.float32).reshape(n, 16, 3), fv)
    sc = synth.Scene(levels=[lv0, lvl], d_thresholds=np.array([d1]), chunk_centers=np.zeros((1, 3)))
    osc = O.OracleScene(sc)
    off = lv0.n
    s_all = np.zeros(n)
    s_clean = np.zeros(n)
    for cam in views:
        g, _, _ = O.active_set(osc, O.MODE_LOD, cam)
        sa, scl = O.importance(osc, cam, g)
        sel = g >= off
        np.maximum.at(s_all, g[sel] - off, sa[sel])
        np.maximum.at(s_clean, g[sel] - off, scl[sel])
    return s_all, s_clean


def test_trained_level_gradients_match_single_level(env):
    """With d_1 = 0 the LOD frame renders all of level 1 and none of level 0,
    so the gradients of the trained level through lodge_render_params_lod
    equal those of the same parameters rendered alone (lodge_render_params,
    whose adjoint is pinned against the FP64 oracle), and the image is the
    same."""
    torch, api = env
    from paper_2505_23158_gb300 import lod_build
    scene = synth.finetune_scene(seed=4, n=20_000)
    cam = synth.finetune_cameras(scene, seed=4, n=1, width=192, height_px=108)[0]
    dev = torch.device("cuda")
    fv = lod_build.filter_variance(0.2, 10.0, cam.fy)
    with api.Lodge(0) as ctx:
        base = lod_build.level_params(scene.levels[0], dev)
        w = torch.randn(cam.height, cam.width, 3, device=dev)
        p1 = [t.clone().requires_grad_(True) for t in base]
        img1 = api.render_level_lod(ctx, p1, [base], 1, cam, [0.0], [0.0, fv])
        (img1 * w).sum().backward()
        p2 = [t.clone().requires_grad_(True) for t in base]
        img2 = api.render_differentiable(ctx, *p2, cam, filter_var=fv)
        (img2 * w).sum().backward()
        assert torch.equal(img1, img2)
        for a, b, name in zip(p1, p2, ["means", "log_scales", "quats", "logits", "sh"]):
            ga, gb = a.grad.double(), b.grad.double()
            rel = float((ga - gb).norm() / max(float(gb.norm()), 1e-30))
            assert rel < 1e-5, (name, rel)
            assert float(gb.norm()) > 0, name


def test_build_level_one(env):
    torch, api = env
    from paper_2505_23158_gb300 import lod_build
    scene = synth.finetune_scene(seed=3, n=30_000)
    views = synth.finetune_cameras(scene, seed=3, n=8, width=160, height_px=96)
    lv0 = scene.levels[0]
    dev = torch.device("cuda")
    d1, gamma = 10.0, 0.02
    fv = lod_build.filter_variance(0.2, d1, views[0].fy)
    with api.Lodge(0) as ctx:
        base = lod_build.level_params(lv0, dev)
        base0 = [t.clone() for t in base]
        targets = [ctx.render_params(*base, cam, save=False)[0] for cam in views]
        g1, hist = lod_build.build_level(ctx, [base], base, [d1], views, targets, gamma, fv, [0.0],
                                         steps=1000, seed=5, keep_params=True)
        for a, b in zip(base, base0):
            assert torch.equal(a, b)                     # level 0 untouched
    assert g1[0].shape[0] == hist[-1]["kept"]
    for rec in hist:
        s_gpu = rec["scores"].astype(np.float64)
        s_all, s_clean = _oracle_scores(lv0, rec["scored_params"], fv, d1, views)
        assert s_gpu.shape == s_all.shape
        lo_bad = s_gpu < s_clean - MARGIN
        hi_bad = s_gpu > s_all + MARGIN
        assert not lo_bad.any() and not hi_bad.any(), (rec["round"], int(lo_bad.sum()), int(hi_bad.sum()))
        thr = rec["threshold"]
        keep_gpu = s_gpu >= thr
        sure_keep = s_clean >= thr + MARGIN
        sure_drop = s_all < thr - MARGIN
        assert keep_gpu[sure_keep].all() and not keep_gpu[sure_drop].any()
        undecided = int((~sure_keep & ~sure_drop).sum())
        first, last = rec["loss_pruned"], rec["loss_tuned"]
        print(f"[build] round {rec['round']}: threshold {thr:.3g}, kept {rec['kept']} of {s_gpu.size}, "
              f"{undecided} within the margin, loss {first:.5f} -> {last:.5f}")
        assert rec["kept"] > 0
        assert last < first, (rec["round"], first, last)
    kept = [r["kept"] for r in hist]
    assert kept[0] >= kept[1] >= kept[2]


def test_render_params_lod_arguments_checked(env):
    """Descending thresholds, a trained level out of range and a saved frame
    that also scores are refused with LODGE_E_INVALID before any work."""
    torch, api = env
    from paper_2505_23158_gb300 import lod_build
    scene = synth.finetune_scene(seed=6, n=2000)
    cam = synth.finetune_cameras(scene, seed=6, n=1, width=64, height_px=48)[0]
    with api.Lodge(0) as ctx:
        base = lod_build.level_params(scene.levels[0], torch.device("cuda"))
        levels = [base, base, base]
        with pytest.raises(api.LodgeError):
            ctx.render_params_lod(levels, cam, [20.0, 10.0], [0.0, 0.0, 0.0])
        with pytest.raises(api.LodgeError):
            ctx.render_params_lod(levels, cam, [10.0, 20.0], [0.0, 0.0, 0.0], train_level=3, save=True)
        score = torch.zeros(3 * base[0].shape[0], device="cuda")
        with pytest.raises(api.LodgeError):
            ctx.render_params_lod(levels, cam, [10.0, 20.0], [0.0, 0.0, 0.0], train_level=1, save=True,
                                  score=score)
        img, st, h = ctx.render_params_lod(levels, cam, [10.0, 20.0], [0.0, 0.0, 0.0])
        assert h is None and img.shape == (48, 64, 3)
