"""GPU adjoint (lodge_render_backward) against the FP64 gradient oracle.

Bars: forward pixels as in the parity tests; gradients within a relative L2
error of 1e-3 per parameter group (FP32 with atomics against FP64)."""
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
    from paper_2505_23158_gb300.api import Lodge
    ctx = Lodge(0)
    yield torch, ctx
    ctx.close()


def _level(n, seed, spread=0.7, log_mean=-2.4):
    rng = np.random.default_rng(seed)
    return synth.Level(rng.uniform(-spread, spread, (n, 3)).astype(np.float32),
                       rng.normal(log_mean, 0.4, (n, 3)).astype(np.float32),
                       rng.normal(size=(n, 4)).astype(np.float32),
                       rng.normal(0.5, 1.0, n).astype(np.float32),
                       rng.normal(0, 0.3, (n, 16, 3)).astype(np.float32))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("seed,n,wh,fv", [(0, 200, (64, 48), 0.0), (1, 400, (80, 60), 0.0),
                                          (2, 150, (33, 47), 0.003)])
def test_gradients_match_fp64_oracle(env, seed, n, wh, fv):
    torch, ctx = env
    from oracle import grad as G
    lv = _level(n, seed)
    cam = synth.look_at((0.1, -0.1, -2.4), (0.0, 0.02, 1.0), (0, -1, 0), wh[0], wh[1], 55.0)
    w = np.random.default_rng(seed + 7).normal(size=(wh[1], wh[0], 3))
    g_ref, img_ref = G.grads(lv, cam, w, filter_var=fv)
    dev = torch.device("cuda")
    ps = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev)
          for a in (lv.means, lv.log_scales, lv.quats, lv.opacity_logits, lv.sh.reshape(n, 48))]
    img, st, h = ctx.render_params(*ps, cam, filter_var=fv, save=True)
    gs = [torch.zeros_like(p) for p in ps]
    ctx.render_backward(h, torch.from_numpy(w.astype(np.float32)).to(dev), *gs)
    ctx.release(h)
    assert np.abs(img.cpu().numpy() - img_ref).max() < 2e-4
    names = ["means", "log_scales", "quats", "opacity_logits", "sh"]
    for name, g, r in zip(names, gs, g_ref):
        e = _rel(g.cpu().numpy().reshape(r.shape).astype(np.float64), r)
        assert e < 1e-3, f"{name}: relative L2 error {e:.3g}"


@pytest.mark.parametrize("seed", [9, 10])
def test_gradients_past_lateral_limits(env, seed):
    """Large Gaussians centred off a narrow (20 degree) view, past the EWA
    Jacobian's lateral limits x/z, y/z = +-1.3 tan(fov/2), reaching into it:
    the clamped Jacobian's forward and adjoint against the FP64 oracle."""
    torch, ctx = env
    from oracle import grad as G
    import oracle as O
    n = 80
    lv = _level(n, seed, spread=1.4, log_mean=-1.0)
    cam = synth.look_at((0.0, 0.0, -2.5), (0.0, 0.0, 1.0), (0, -1, 0), 48, 40, 20.0)
    p = lv.means.astype(np.float64) @ cam.R.astype(np.float64).T + cam.t
    past = ((np.abs(p[:, 0] / p[:, 2]) > 1.3 * cam.width / (2.0 * cam.fx))
            | (np.abs(p[:, 1] / p[:, 2]) > 1.3 * cam.height / (2.0 * cam.fy)))
    sc = synth.Scene(levels=[lv], d_thresholds=np.zeros(0), chunk_centers=np.zeros((1, 3)))
    vis = O.project(O.OracleScene(sc), cam, np.arange(n))["visible"]
    assert (past & vis).sum() >= 10
    w = np.random.default_rng(seed + 7).normal(size=(cam.height, cam.width, 3))
    g_ref, img_ref = G.grads(lv, cam, w)
    dev = torch.device("cuda")
    ps = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev)
          for a in (lv.means, lv.log_scales, lv.quats, lv.opacity_logits, lv.sh.reshape(n, 48))]
    img, st, h = ctx.render_params(*ps, cam, save=True)
    gs = [torch.zeros_like(q) for q in ps]
    ctx.render_backward(h, torch.from_numpy(w.astype(np.float32)).to(dev), *gs)
    ctx.release(h)
    assert np.abs(img.cpu().numpy() - img_ref).max() < 2e-4
    for name, g, r in zip(["means", "log_scales", "quats", "opacity_logits", "sh"], gs, g_ref):
        e = _rel(g.cpu().numpy().reshape(r.shape).astype(np.float64), r)
        assert e < 1e-3, f"{name}: relative L2 error {e:.3g}"


def test_autograd_function_and_fit_step(env):
    """The torch.autograd.Function wrapper gives the same gradients as the
    raw calls, and a few Adam steps lower an L1 loss against a perturbed
    target (the fine-tuning use)."""
    torch, ctx = env
    from paper_2505_23158_gb300.api import render_differentiable
    lv = _level(300, 5)
    cam = synth.look_at((0.0, 0.0, -2.4), (0.0, 0.0, 1.0), (0, -1, 0), 64, 64, 55.0)
    dev = torch.device("cuda")
    target_lv = synth.perturb_scene(synth.Scene(levels=[lv], d_thresholds=np.zeros(0),
                                                chunk_centers=np.zeros((1, 3))), 3,
                                    mean_std=0.02, logit_std=0.3).levels[0]
    tps = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev)
           for a in (target_lv.means, target_lv.log_scales, target_lv.quats,
                     target_lv.opacity_logits, target_lv.sh.reshape(300, 48))]
    with torch.no_grad():
        target, _, h = ctx.render_params(*tps, cam, save=False)
    ps = [torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev).requires_grad_(True)
          for a in (lv.means, lv.log_scales, lv.quats, lv.opacity_logits, lv.sh.reshape(300, 48))]
    opt = torch.optim.Adam(ps, lr=2e-3)
    losses = []
    for it in range(30):
        opt.zero_grad()
        img = render_differentiable(ctx, *ps, cam)
        loss = (img - target).abs().mean()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.8 * losses[0], losses
