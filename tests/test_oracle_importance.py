"""Pins of the oracle's importance score (Sec. 3, "Importance pruning" and
"Visibility filtering", after RadSplat: the largest blending weight
T * alpha a Gaussian receives at any pixel of the views).

Checked against closed forms (one and two Gaussians on the optical axis), the
rendered image (with a single Gaussian coloured white and every other one
black, each pixel of the render is that Gaussian's weight there), and
invariants (occluded and culled Gaussians score 0, scores never exceed the
alpha clamp, views accumulate by maximum)."""
import math

import numpy as np

import pytest

import oracle as O
from paper_2505_23158_gb300 import synth


@pytest.fixture(scope="module")
def small_plain():
    return synth.plain_scene(0), synth.plain_camera(64, 64)


def _scene(means, log_scales, logits, sh):
    n = len(means)
    lvl = synth.Level(np.asarray(means, np.float32), np.asarray(log_scales, np.float32),
                      np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
                      np.asarray(logits, np.float32), np.asarray(sh, np.float32))
    return synth.Scene(levels=[lvl], d_thresholds=np.zeros(0), chunk_centers=np.zeros((1, 3)))


def _sh(rgb):
    sh = np.zeros((16, 3), np.float32)
    sh[0] = (np.asarray(rgb, np.float64) - 0.5) / (0.5 / math.sqrt(math.pi))
    return sh


def _f32_act(log_s, logit):
    s = float(np.float32(math.exp(np.float32(log_s))))
    o = float(np.float32(1 / (1 + math.exp(-np.float32(logit)))))
    return s, o


def test_single_gaussian_closed_form():
    """T = 1 at every pixel, so the score is o exp(-1/2 d^2 / sigma'^2) at the
    pixel centre nearest the projected mean: with the mean on a pixel corner,
    d^2 = 0.5 and sigma'^2 = fx^2 s^2 / z^2 + 0.3."""
    log_s, logit = math.log(0.05), math.log(0.8 / 0.2)
    sc = _scene([[0, 0, 0]], [[log_s] * 3], [logit], [_sh((1, 1, 1))])
    cam = synth.plain_camera(64, 64)          # camera at z = -3, cx = cy = 32
    score, clean = O.importance(O.OracleScene(sc), cam, np.arange(1))
    s, o = _f32_act(log_s, logit)
    var = cam.fx ** 2 * s ** 2 / 9.0 + 0.3
    expect = o * math.exp(-0.5 * 0.5 / var)
    assert abs(score[0] - expect) < 1e-7
    assert clean[0] == score[0]


def test_two_gaussians_closed_form():
    """Front Gaussian 1 and back Gaussian 2, both on the axis: the back one's
    weight at a pixel is (1 - alpha1) alpha2.  With G the pixel's Gaussian
    factor of each, the score is the maximum over pixels of
    (1 - o1 G1) o2 G2, evaluated here pixel by pixel from the closed form."""
    l1, l2 = math.log(0.2), math.log(0.3)
    g1, g2 = math.log(0.3 / 0.7), math.log(0.7 / 0.3)
    sc = _scene([[0, 0, -1.0], [0, 0, 1.0]], [[l1] * 3, [l2] * 3], [g1, g2],
                [_sh((1, 0, 0)), _sh((0, 1, 0))])
    cam = synth.plain_camera(32, 32)
    score, _ = O.importance(O.OracleScene(sc), cam, np.arange(2))
    s1, o1 = _f32_act(l1, g1)
    s2, o2 = _f32_act(l2, g2)
    v1 = cam.fx ** 2 * s1 ** 2 / 4.0 + 0.3
    v2 = cam.fx ** 2 * s2 ** 2 / 16.0 + 0.3
    ys, xs = np.mgrid[0:32, 0:32]
    d2 = (xs + 0.5 - cam.cx) ** 2 + (ys + 0.5 - cam.cy) ** 2
    a1 = np.minimum(0.99, o1 * np.exp(-0.5 * d2 / v1))
    a2 = np.minimum(0.99, o2 * np.exp(-0.5 * d2 / v2))
    a1 = np.where(a1 >= 1 / 255, a1, 0.0)
    w2 = np.where(a2 >= 1 / 255, (1 - a1) * a2, 0.0)
    assert abs(score[0] - a1.max()) < 1e-7
    assert abs(score[1] - w2.max()) < 1e-7


def test_score_is_max_of_masked_render(small_plain):
    """Colour one Gaussian white and all others black: the rendered image is
    that Gaussian's weight at each pixel, so its score is the image maximum."""
    sc, cam = small_plain
    osc = O.OracleScene(sc)
    score, _ = O.importance(osc, cam, np.arange(sc.n_total))
    picks = np.argsort(-score)[[0, 5, 50, 300]]
    lv = sc.levels[0]
    for i in picks:
        sh = np.zeros_like(lv.sh)
        sh[:, 0, :] = -0.5 / (0.5 / math.sqrt(math.pi))   # rgb = max(0, 0) = 0
        sh[i, 0, :] = 0.5 / (0.5 / math.sqrt(math.pi))    # rgb = 1
        masked = synth.Scene(levels=[synth.Level(lv.means, lv.log_scales, lv.quats,
                                                 lv.opacity_logits, sh)],
                             d_thresholds=np.zeros(0), chunk_centers=np.zeros((1, 3)))
        img = O.render(O.OracleScene(masked), cam, np.arange(sc.n_total))["rgb"]
        assert abs(img[..., 0].max() - score[i]) < 1e-6, i


def test_occluded_and_culled_score_zero():
    """An opaque stack ends every pixel after two Gaussians (wide enough that
    alpha is clamped at 0.99 on the whole 16x16 image): the ones behind score
    0, as does one behind the camera."""
    n = 4
    means = [[0, 0, 0.5 * i] for i in range(n)] + [[0, 0, -10.0]]
    sc = _scene(means, [[math.log(50.0)] * 3] * (n + 1), [12.0] * (n + 1),
                [_sh((1, 1, 1))] * (n + 1))
    cam = synth.plain_camera(16, 16)
    score, _ = O.importance(O.OracleScene(sc), cam, np.arange(n + 1))
    assert score[0] == 0.99 and abs(score[1] - 0.01 * 0.99) < 1e-15
    assert score[2] == 0.0 and score[3] == 0.0 and score[4] == 0.0


def test_bounds(small_plain):
    sc, cam = small_plain
    s1, c1 = O.importance(O.OracleScene(sc), cam, np.arange(sc.n_total))
    assert (s1 >= 0).all() and (s1 <= 0.99).all() and (c1 <= s1).all()
    assert (s1 > 0).sum() > 100
