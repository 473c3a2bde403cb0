"""Pins of the oracle's knife-edge enumeration and of the pixel comparison.

Eq. 1 makes two discrete decisions per pair: skip alpha < 1/255 and stop
before T drops below 1e-4.  Where the FP32 error bound of the compared
value spans the threshold, the FP32 renderer may take either branch and both
renders are correct; the oracle reports the range of results over all such
choices.  These tests pin that range to closed forms on one and two
Gaussians and to the opaque stack whose transmittance lands on 1e-4, and
plant mistakes in an image to check the comparison rejects them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2505_23158_gb300 import synth


def _scene(means, log_scales, logits, rgbs):
    n = len(means)
    y00 = 0.5 / math.sqrt(math.pi)
    sh = np.zeros((n, 16, 3), np.float32)
    for i, c in enumerate(rgbs):
        sh[i, 0] = (np.asarray(c, np.float64) - 0.5) / y00
    lvl = synth.Level(np.asarray(means, np.float32), np.asarray(log_scales, np.float32),
                      np.asarray([[1, 0, 0, 0]] * n, np.float32), np.asarray(logits, np.float32),
                      sh, 0.0)
    return synth.Scene(levels=[lvl], d_thresholds=np.zeros(0), chunk_centers=np.zeros((1, 3)))


def _f32_sigma(sigma):
    return float(np.float32(math.exp(np.float32(math.log(sigma)))))


def _f32_opacity(logit):
    return float(np.float32(1 / (1 + math.exp(-float(np.float32(logit))))))


def _logit_for(o):
    return math.log(o / (1 - o))


def _grid(cam):
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    return (xs + 0.5 - cam.cx) ** 2 + (ys + 0.5 - cam.cy) ** 2


@pytest.mark.parametrize("delta", [3e-4, -3e-4])
def test_alpha_skip_knife_closed_form(delta):
    """One isotropic Gaussian on the axis (Sigma' = v I) whose alpha at pixel
    (37, 32) is (1/255)(1 + delta): that pixel is a knife edge, and so is
    every pixel whose alpha lies within the error bound e = (d / v) dd + ke0
    of 1/255.  At a knife pixel the two renders are 0 (skipped) and alpha rgb
    (blended); elsewhere the single closed-form render."""
    cam = synth.plain_camera(64, 64)
    sigma, z = 0.1, 3.0
    s = _f32_sigma(sigma)
    v = cam.fx ** 2 * s ** 2 / z ** 2 + 0.3
    d2_target = (37.5 - cam.cx) ** 2 + (32.5 - cam.cy) ** 2
    o = (1 / 255) * (1 + delta) * math.exp(0.5 * d2_target / v)
    rgb = np.array([0.9, 0.5, 0.2])
    sc = _scene([[0, 0, 0]], [[math.log(sigma)] * 3], [_logit_for(o)], [rgb])
    r = O.render(O.OracleScene(sc), cam, np.arange(1))
    oe = _f32_opacity(np.float32(_logit_for(o)))
    d2 = _grid(cam)
    a = np.minimum(0.99, oe * np.exp(-0.5 * d2 / v))
    e = np.sqrt(d2) / v * O.ERR_DD + O.ERR_KE0
    knife = np.abs(a - 1 / 255) <= e / 255
    assert knife[32, 37]
    assert np.array_equal(r["knife_code"] == 1, knife) and not (r["knife_code"] == 2).any()
    kept = np.where(a >= 1 / 255, a, 0.0)[..., None] * rgb
    assert np.abs(r["rgb"] - kept).max() < 1e-6
    lo = np.where(knife[..., None], 0.0, kept)
    hi = np.where(knife[..., None], a[..., None] * rgb, kept)
    assert np.abs(r["lo"] - lo).max() < 1e-6 and np.abs(r["hi"] - hi).max() < 1e-6
    # with a zero error bound no decision is a knife edge
    r0 = O.render(O.OracleScene(sc), cam, np.arange(1), err_dd=0.0, err_ke0=0.0)
    assert not r0["knife_code"].any()
    assert np.array_equal(r0["lo"], r0["rgb"]) and np.array_equal(r0["hi"], r0["rgb"])
    assert np.array_equal(r0["rgb"], r["rgb"])


def test_transmittance_stop_knife_on_opaque_stack():
    """Four large opaque Gaussians on the axis: alpha is clamped to 0.99 at
    the centre, so T after two is 0.01^2, which is 1e-4 up to rounding.  The
    oracle stops before the third (FP64 puts T just above 1e-4); an FP32
    renderer may stop before the second.  Both are in the range: the
    channel lies in [0.99 c, (0.99 + 0.01 0.99) c]."""
    n = 4
    means = [[0, 0, 0.5 * i] for i in range(n)]
    sc = _scene(means, [[math.log(5.0)] * 3] * n, [12.0] * n, [(1, 1, 1)] * n)
    cam = synth.plain_camera(16, 16)
    r = O.render(O.OracleScene(sc), cam, np.arange(n))
    col = r["rgb"][8, 8, 0] / (0.99 + 0.01 * 0.99)
    assert abs(col - 1) < 1e-6
    assert r["knife_code"][8, 8] == 1 and r["ncontrib"][8, 8] == 2
    assert abs(r["lo"][8, 8, 0] - 0.99 * col) < 1e-12
    assert abs(r["hi"][8, 8, 0] - (0.99 + 0.01 * 0.99) * col) < 1e-12


def test_two_knife_decisions_enumerate_every_path():
    """Two Gaussians on the axis, each at alpha = (1/255)(1 + 3e-4) at pixel
    (37, 32), colours (1,0,0) in front and (1,1,0) behind.  The four paths
    give channel 0 in {a1 + (1-a1) a2, a2, a1, 0} and channel 1 in
    {(1-a1) a2, a2, a1 ... 0}: the lower bound 0 of channel 0 needs both
    decisions flipped, the upper bound a2 of channel 1 needs only the
    front one flipped."""
    cam = synth.plain_camera(64, 64)
    sig = [0.1, 0.12]
    zs = [0.0, 1.0]
    px, py = 37, 32
    d2_target = (px + 0.5 - cam.cx) ** 2 + (py + 0.5 - cam.cy) ** 2
    logits, alphas = [], []
    for sg, mz in zip(sig, zs):
        v = cam.fx ** 2 * _f32_sigma(sg) ** 2 / (3.0 + mz) ** 2 + 0.3
        o = (1 / 255) * (1 + 3e-4) * math.exp(0.5 * d2_target / v)
        assert o < 1
        lg = _logit_for(o)
        logits.append(lg)
        alphas.append(_f32_opacity(np.float32(lg)) * math.exp(-0.5 * d2_target / v))
    a1, a2 = alphas
    sc = _scene([[0, 0, zs[0]], [0, 0, zs[1]]], [[math.log(sig[0])] * 3, [math.log(sig[1])] * 3],
                logits, [(1, 0, 0), (1, 1, 0)])
    r = O.render(O.OracleScene(sc), cam, np.arange(2))
    assert r["knife_code"][py, px] == 1
    assert abs(r["rgb"][py, px, 0] - (a1 + (1 - a1) * a2)) < 1e-6
    assert abs(r["lo"][py, px, 0]) < 1e-6
    assert abs(r["hi"][py, px, 0] - (a1 + (1 - a1) * a2)) < 1e-6
    assert abs(r["lo"][py, px, 1]) < 1e-6
    assert abs(r["hi"][py, px, 1] - a2) < 1e-6


def test_compare_pixels_rejects_planted_mistakes():
    """The comparison passes the oracle's own image and any image inside the
    knife-edge ranges, and rejects a non-knife pixel off by 3e-4, a knife
    pixel 3e-4 outside its range, and a small bias on every pixel (mean)."""
    scene, cams = synth.workload_plain(0)
    osc = O.OracleScene(scene)
    cam = synth.plain_camera(96, 96)
    ref = O.render(osc, cam, np.arange(osc.n_total))
    img = ref["rgb"].astype(np.float32)
    out = O.compare_pixels(img, ref)
    assert out["max_abs"] < 1e-6 and out["unresolved"] == 0
    code = ref["knife_code"]
    assert (code == 1).any(), "workload has no knife-edge pixel to plant in"
    ky, kx = np.argwhere(code == 1)[0]
    alt = img.copy()
    alt[code == 1] = np.clip(ref["lo"], 0, 1)[code == 1]
    assert O.compare_pixels(alt, ref)["knife"] == int((code > 0).sum())
    ny, nx = np.argwhere((code == 0) & (ref["rgb"].max(axis=2) > 0.1) & (ref["rgb"].max(axis=2) < 0.9))[0]
    bad = img.copy(); bad[ny, nx, 1] += 3e-4
    with pytest.raises(AssertionError):
        O.compare_pixels(bad, ref)
    bad = img.copy()
    lo_c = np.clip(ref["lo"][ky, kx], 0, 1)
    c = int(np.argmax(lo_c > 1e-3)) if (lo_c > 1e-3).any() else 0
    bad[ky, kx, c] = max(0.0, lo_c[c] - 3e-4) if lo_c[c] > 3e-4 else np.clip(ref["hi"][ky, kx, c], 0, 1) + 3e-4
    with pytest.raises(AssertionError):
        O.compare_pixels(bad, ref)
    with pytest.raises(AssertionError):
        O.compare_pixels(img + 2e-5, ref)
