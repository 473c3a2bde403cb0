"""Pins of the FP64 gradient oracle (oracle/grad.py).

Its forward must equal oracle.c's render (an independent implementation of
the same definition), and its autograd gradients must equal central finite
differences of that forward (h = 1e-4 scaled), for every parameter whose
perturbation leaves the discrete decisions (1/255 skip, T < 1e-4 stop)
unchanged.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
from oracle import grad as G
from paper_2505_23158_gb300 import synth


def _scene(n, seed, spread=0.6, log_mean=-2.2):
    rng = np.random.default_rng(seed)
    lvl = synth.Level(rng.uniform(-spread, spread, (n, 3)).astype(np.float32),
                      rng.normal(log_mean, 0.4, (n, 3)).astype(np.float32),
                      rng.normal(size=(n, 4)).astype(np.float32),
                      rng.normal(0.5, 1.0, n).astype(np.float32),
                      rng.normal(0, 0.3, (n, 16, 3)).astype(np.float32))
    return synth.Scene(levels=[lvl], d_thresholds=np.zeros(0), chunk_centers=np.zeros((1, 3)))


def test_torch_forward_equals_c_oracle():
    sc = _scene(300, 1)
    cam = synth.look_at((0.2, -0.1, -2.5), (0.0, 0.05, 1.0), (0, -1, 0), 64, 48, 55.0)
    ref = O.render(O.OracleScene(sc), cam, np.arange(300))
    lv = sc.levels[0]
    with torch.no_grad():
        img, T, nc, _ = G.render_t(*G.params_t(lv, False), cam, return_aux=True)
    # oracle.c rounds the FP64 activations to FP32 once; this forward keeps
    # them in FP64, so the two agree to FP32 rounding of the parameters
    ok = ~ref["knife"]
    assert np.abs(img.numpy() - ref["rgb"])[ok].max() < 2e-6
    assert np.abs(T.numpy() - ref["T"])[ok].max() < 2e-6
    assert (nc.numpy()[ok].astype(np.int32) != ref["ncontrib"][ok]).mean() < 1e-3


def test_torch_forward_with_filter_and_multipliers():
    sc = _scene(120, 2)
    sc.levels[0].filter_var = 0.004
    cam = synth.look_at((0.0, 0.0, -2.5), (0.0, 0.0, 1.0), (0, -1, 0), 40, 40, 55.0)
    mults = np.random.default_rng(3).uniform(0.2, 1.0, 120).astype(np.float32)
    ref = O.render(O.OracleScene(sc), cam, np.arange(120), mults)
    with torch.no_grad():
        img = G.render_t(*G.params_t(sc.levels[0], False), cam, mults=mults,
                         filter_var=0.004)
    ok = ~ref["knife"]
    assert np.abs(img.numpy() - ref["rgb"])[ok].max() < 2e-6


@pytest.mark.parametrize("seed", [11, 12])
def test_autograd_matches_central_differences(seed):
    sc = _scene(12, seed, spread=0.35, log_mean=-1.8)
    cam = synth.look_at((0.05, -0.05, -2.0), (0.0, 0.0, 1.0), (0, -1, 0), 20, 16, 50.0)
    _check_fd(sc, cam, seed, 60)


def _lateral(sc, cam):
    """x/z and y/z of each Gaussian's camera point against the Jacobian's
    lateral limits 1.3 W / (2 fx), 1.3 H / (2 fy): how many of the visible
    Gaussians lie past them."""
    p = sc.levels[0].means.astype(np.float64) @ cam.R.astype(np.float64).T + cam.t
    limx = 1.3 * cam.width / (2.0 * cam.fx)
    limy = 1.3 * cam.height / (2.0 * cam.fy)
    past = (np.abs(p[:, 0] / p[:, 2]) > limx) | (np.abs(p[:, 1] / p[:, 2]) > limy)
    vis = O.project(O.OracleScene(sc), cam, np.arange(sc.levels[0].n))["visible"]
    return int((past & vis).sum())


@pytest.mark.parametrize("seed", [21, 22])
def test_autograd_past_lateral_limits(seed):
    """Large Gaussians centred off the image, past the Jacobian's lateral
    limits, reaching into a narrow (20 degree) view: the forward equals
    oracle.c's, and the gradients through the clamped Jacobian (no x/z
    derivative of its third column) equal central differences."""
    sc = _scene(12, seed, spread=1.4, log_mean=-1.0)
    cam = synth.look_at((0.0, 0.0, -2.5), (0.0, 0.0, 1.0), (0, -1, 0), 20, 16, 20.0)
    assert _lateral(sc, cam) >= 5
    ref = O.render(O.OracleScene(sc), cam, np.arange(12))
    with torch.no_grad():
        img = G.render_t(*G.params_t(sc.levels[0], False), cam)
    ok = ~ref["knife"]
    assert np.abs(img.numpy() - ref["rgb"])[ok].max() < 2e-6
    _check_fd(sc, cam, seed, 40)


def _check_fd(sc, cam, seed, min_checked):
    lv = sc.levels[0]
    w = np.random.default_rng(seed).normal(size=(cam.height, cam.width, 3))
    grads, _ = G.grads(lv, cam, w)
    base = [np.asarray(a, np.float32).astype(np.float64) for a in
            (lv.means, lv.log_scales, lv.quats, lv.opacity_logits, lv.sh)]
    wt = torch.as_tensor(w)

    def f(vals):
        with torch.no_grad():
            ts = [torch.as_tensor(v) for v in vals]
            img, _, _, sig = G.render_t(*ts, cam, return_aux=True)
            return float((img * wt).sum()), sig

    _, sig0 = f(base)
    rng = np.random.default_rng(seed + 100)
    checked = 0
    for gi, g in enumerate(grads):
        flat = base[gi].reshape(-1)
        picks = rng.choice(flat.size, size=min(flat.size, 24), replace=False)
        for j in picks:
            h = 1e-4 * max(1.0, abs(flat[j]))
            vp = [b.copy() for b in base]; vm = [b.copy() for b in base]
            vp[gi].reshape(-1)[j] += h
            vm[gi].reshape(-1)[j] -= h
            fp, sp = f(vp)
            fm, sm = f(vm)
            if sp != sig0 or sm != sig0:
                continue   # a discrete decision flipped: FD is not a derivative here
            fd = (fp - fm) / (2 * h)
            an = g.reshape(-1)[j]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-7, (gi, j, fd, an)
            checked += 1
    assert checked >= min_checked
    for g in grads:
        assert np.abs(g).max() > 0
