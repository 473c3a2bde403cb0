"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed
form, brute force, an invariant, a textbook special case.  Tests are chosen so
that a plausible slip (a dropped term, a wrong sign or index, a transposed
operand) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2505_23158_gb300 import synth


def _single_level_scene(means, log_scales, quats, logits, sh, filter_var=0.0):
    lvl = synth.Level(np.asarray(means, np.float32), np.asarray(log_scales, np.float32),
                      np.asarray(quats, np.float32), np.asarray(logits, np.float32),
                      np.asarray(sh, np.float32), filter_var)
    return synth.Scene(levels=[lvl], d_thresholds=np.zeros(0), chunk_centers=np.zeros((1, 3)))


def _sh_for_rgb(rgb):
    """Degree-0 coefficients giving the colour rgb (Y00 = 1/(2 sqrt(pi)))."""
    y00 = 0.5 / math.sqrt(math.pi)
    sh = np.zeros((16, 3), np.float32)
    sh[0] = (np.asarray(rgb, np.float64) - 0.5) / y00
    return sh


def _logit(o):
    return math.log(o / (1 - o))


# --------------------------------------------------------------------------
# Eq. 1 compositing: closed forms
# --------------------------------------------------------------------------
def test_single_isotropic_gaussian_closed_form():
    """A single isotropic Gaussian of std sigma on the optical axis at depth z
    projects to Sigma' = (fx^2 sigma^2 / z^2 + 0.3) I; each pixel equals
    o exp(-1/2 d^T Sigma'^-1 d) rgb wherever that alpha >= 1/255."""
    sigma, z, o = 0.05, 3.0, 0.8
    rgb = (0.9, 0.4, 0.2)
    sc = _single_level_scene([[0, 0, 0]], [[math.log(sigma)] * 3], [[1, 0, 0, 0]],
                             [_logit(o)], [_sh_for_rgb(rgb)])
    cam = synth.plain_camera(64, 64)
    osc = O.OracleScene(sc)
    r = O.render(osc, cam, np.arange(1))
    s_eff = float(np.float32(math.exp(np.float32(math.log(sigma)))))  # FP32 activated
    var = cam.fx ** 2 * s_eff ** 2 / z ** 2 + 0.3
    ys, xs = np.mgrid[0:64, 0:64]
    d2 = (xs + 0.5 - cam.cx) ** 2 + (ys + 0.5 - cam.cy) ** 2
    o_eff = float(np.float32(1 / (1 + math.exp(-np.float32(_logit(o))))))
    a = np.minimum(0.99, o_eff * np.exp(-0.5 * d2 / var))
    a = np.where(a >= 1 / 255, a, 0.0)
    expect = a[..., None] * np.asarray(rgb)[None, None, :]
    assert np.abs(r["rgb"] - expect).max() < 1e-6
    assert np.abs(r["T"] - (1 - a)).max() < 1e-12
    assert (r["ncontrib"] == (a > 0)).all()


def test_single_gaussian_with_compensated_2d_filter():
    """Mip-Splatting's 2D filter (supplementary "Details on training the full
    representation"): with Sigma2D = s^2 I (s = fx sigma / z), Sigma' = (s^2 +
    0.3) I and the opacity is scaled by sqrt(det Sigma2D / det Sigma') =
    s^2 / (s^2 + 0.3), so each pixel is o s^2/(s^2+0.3) exp(-d^2 / (2 (s^2 +
    0.3))) rgb, and the splat's integral no longer depends on the 0.3."""
    sigma, z, o = 0.01, 3.0, 0.8
    rgb = (0.9, 0.4, 0.2)
    sc = _single_level_scene([[0, 0, 0]], [[math.log(sigma)] * 3], [[1, 0, 0, 0]],
                             [_logit(o)], [_sh_for_rgb(rgb)])
    sc.filter2d = True
    cam = synth.plain_camera(64, 64)
    r = O.render(O.OracleScene(sc), cam, np.arange(1))
    s_eff = float(np.float32(math.exp(np.float32(math.log(sigma)))))
    s2 = cam.fx ** 2 * s_eff ** 2 / z ** 2
    o_eff = float(np.float32(1 / (1 + math.exp(-np.float32(_logit(o))))))
    ys, xs = np.mgrid[0:64, 0:64]
    d2 = (xs + 0.5 - cam.cx) ** 2 + (ys + 0.5 - cam.cy) ** 2
    a = np.minimum(0.99, o_eff * s2 / (s2 + 0.3) * np.exp(-0.5 * d2 / (s2 + 0.3)))
    a = np.where(a >= 1 / 255, a, 0.0)
    assert np.abs(r["rgb"] - a[..., None] * np.asarray(rgb)).max() < 1e-6
    # integral: o * 2 pi s^2 with the filter, o * 2 pi (s^2 + 0.3) without
    plain = O.render(O.OracleScene(_single_level_scene([[0, 0, 0]], [[math.log(sigma)] * 3],
                                                       [[1, 0, 0, 0]], [_logit(o)],
                                                       [_sh_for_rgb(rgb)])), cam, np.arange(1))
    ratio = r["rgb"][..., 0].sum() / plain["rgb"][..., 0].sum()
    assert abs(ratio - s2 / (s2 + 0.3)) < 0.02


def test_two_gaussians_closed_form():
    """Two Gaussians on the axis: front alpha1 c1 + (1 - alpha1) alpha2 c2,
    the nearer one in front regardless of input order."""
    s1, s2 = 0.2, 0.3
    o1, o2 = 0.6, 0.7
    c1, c2 = (1.0, 0.0, 0.0), (0.0, 1.0, 0.0)
    for order in ((0, 1), (1, 0)):
        means = np.array([[0, 0, -1.0], [0, 0, 1.0]])[list(order)]
        ls = np.log(np.array([[s1] * 3, [s2] * 3]))[list(order)]
        lg = np.array([_logit(o1), _logit(o2)])[list(order)]
        sh = np.stack([_sh_for_rgb(c1), _sh_for_rgb(c2)])[list(order)]
        sc = _single_level_scene(means, ls, [[1, 0, 0, 0]] * 2, lg, sh)
        cam = synth.plain_camera(32, 32)
        r = O.render(O.OracleScene(sc), cam, np.arange(2))
        px = 16  # pixel (16,16) has centre (16.5, 16.5); cx = 16
        d2 = 0.5 ** 2 * 2
        e1 = float(np.float32(math.exp(np.float32(math.log(s1)))))
        e2 = float(np.float32(math.exp(np.float32(math.log(s2)))))
        v1 = cam.fx ** 2 * e1 ** 2 / 2.0 ** 2 + 0.3
        v2 = cam.fx ** 2 * e2 ** 2 / 4.0 ** 2 + 0.3
        oe1 = float(np.float32(1 / (1 + math.exp(-np.float32(_logit(o1))))))
        oe2 = float(np.float32(1 / (1 + math.exp(-np.float32(_logit(o2))))))
        a1 = oe1 * math.exp(-0.5 * d2 / v1)
        a2 = oe2 * math.exp(-0.5 * d2 / v2)
        expect = a1 * np.array(c1) + (1 - a1) * a2 * np.array(c2)
        assert np.abs(r["rgb"][px, px] - expect).max() < 1e-6
        assert abs(r["T"][px, px] - (1 - a1) * (1 - a2)) < 1e-12


def test_alpha_clamp_and_termination():
    """Opaque stack: alpha is clamped at 0.99, so T after k Gaussians is
    0.01^k; the third would drop T below 1e-4 and is not blended."""
    n = 4
    means = np.array([[0, 0, 0.5 * i] for i in range(n)], np.float64)
    sc = _single_level_scene(means, np.full((n, 3), math.log(5.0)), [[1, 0, 0, 0]] * n,
                             [12.0] * n, [_sh_for_rgb((1, 1, 1))] * n)
    cam = synth.plain_camera(16, 16)
    r = O.render(O.OracleScene(sc), cam, np.arange(n))
    # large Gaussians: o G > 0.99 at the centre pixel, so alpha = 0.99 for all
    # four; (1 - 0.99)^2 rounds just above 1e-4 in FP64, (1 - 0.99)^3 < 1e-4
    assert r["ncontrib"][8, 8] == 2
    assert r["T"][8, 8] == (1 - 0.99) * (1 - 0.99)
    assert abs(r["rgb"][8, 8, 0] - (0.99 + 0.01 * 0.99)) < 1e-7  # FP32 SH coefficient


# --------------------------------------------------------------------------
# sorting, binning and transmittance: brute force and invariants
# --------------------------------------------------------------------------
def test_binned_equals_brute_force(plain):
    """Brute force (every Gaussian at every pixel, one global depth sort)
    equals the 16x16-tile binned render; this pins the tile rect as
    conservative for the 1/255 skip and the per-tile sort."""
    scene, cams, osc = plain
    g = np.arange(osc.n_total)
    cam = synth.plain_camera(64, 64)
    rb = O.render(osc, cam, g, brute=True)
    rt = O.render(osc, cam, g)
    assert np.array_equal(rb["rgb"], rt["rgb"])
    assert np.array_equal(rb["T"], rt["T"])
    assert np.array_equal(rb["ncontrib"], rt["ncontrib"])


def test_binned_equals_brute_force_random_small():
    rng = np.random.default_rng(7)
    for trial in range(3):
        n = 300
        sc = _single_level_scene(rng.uniform(-1, 1, (n, 3)), rng.normal(-2.5, 0.7, (n, 3)),
                                 rng.normal(size=(n, 4)), rng.normal(0, 2, n),
                                 rng.normal(0, 0.3, (n, 16, 3)))
        cam = synth.look_at((0.3, -0.2, -2.5), (0.05, 0.1, 1.0), (0, -1, 0), 48, 40, 55.0)
        osc = O.OracleScene(sc)
        g = np.arange(n)
        rb = O.render(osc, cam, g, brute=True)
        rt = O.render(osc, cam, g)
        assert np.array_equal(rb["rgb"], rt["rgb"]), trial


def test_permutation_invariance(plain):
    """Permuting the input leaves the image unchanged wherever no two
    Gaussians share an FP32 depth (tied depths are ordered by record, which
    moves with the permutation; their tiles are excluded)."""
    scene, cams, osc = plain
    cam = cams[0]
    r0 = O.render(osc, cam, np.arange(osc.n_total))
    perm = np.random.default_rng(3).permutation(osc.n_total)
    lv = scene.levels[0]
    sc2 = _single_level_scene(lv.means[perm], lv.log_scales[perm], lv.quats[perm],
                              lv.opacity_logits[perm], lv.sh[perm])
    osc2 = O.OracleScene(sc2)
    r1 = O.render(osc2, cam, np.arange(osc.n_total))
    pr = O.project(osc, cam, np.arange(osc.n_total))
    vis = np.flatnonzero(pr["visible"])
    zs = pr["z"][vis]
    _, inv, cnt = np.unique(zs, return_inverse=True, return_counts=True)
    tied = vis[cnt[inv] > 1]
    mask = np.ones((cam.height, cam.width), bool)
    for i in tied:
        x0, y0, x1, y1 = pr["rect"][i]
        mask[y0 * 16:(y1 + 1) * 16, x0 * 16:(x1 + 1) * 16] = False
    assert mask.mean() > 0.5
    assert np.abs(r0["rgb"] - r1["rgb"])[mask].max() < 1e-12


def test_tie_break_by_record_order():
    """Two Gaussians at the same FP32 depth: the lower record composites
    first."""
    means = [[0, 0, 0], [0, 0, 0]]
    sc = _single_level_scene(means, [[math.log(0.3)] * 3] * 2, [[1, 0, 0, 0]] * 2,
                             [_logit(0.5)] * 2, [_sh_for_rgb((1, 0, 0)), _sh_for_rgb((0, 0, 1))])
    cam = synth.plain_camera(16, 16)
    r = O.render(O.OracleScene(sc), cam, np.arange(2))
    red, blue = r["rgb"][8, 8, 0], r["rgb"][8, 8, 2]
    assert red > blue  # first record in front


def test_unit_colour_weights_telescope(plain):
    """With every colour equal to 1, C = sum T_i alpha_i = 1 - T_final
    (the blend weights telescope)."""
    scene, cams, _ = plain
    lv = scene.levels[0]
    sh = np.zeros_like(lv.sh)
    sh[:, 0, :] = _sh_for_rgb((1, 1, 1))[0]
    sc = _single_level_scene(lv.means, lv.log_scales, lv.quats, lv.opacity_logits, sh)
    r = O.render(O.OracleScene(sc), cams[0], np.arange(lv.n))
    col = float(sh[0, 0, 0]) * (0.5 / math.sqrt(math.pi)) + 0.5  # 1 up to FP32 rounding
    for c in range(3):
        assert np.abs(r["rgb"][..., c] - col * (1 - r["T"])).max() < 1e-12
    assert r["T"].min() >= 1e-4 and r["T"].max() <= 1.0


def test_zero_opacity_gives_background(plain):
    scene, cams, _ = plain
    lv = scene.levels[0]
    sc = _single_level_scene(lv.means, lv.log_scales, lv.quats,
                             np.full(lv.n, -200.0), lv.sh)
    r = O.render(O.OracleScene(sc), cams[0], np.arange(lv.n))
    assert np.all(r["rgb"] == 0) and np.all(r["T"] == 1) and r["n_keys"] == 0


def test_keys_sorted_and_match_rects(plain):
    scene, cams, osc = plain
    k, g = O.keys(osc, cams[0], np.arange(osc.n_total))
    assert np.all(np.diff(k.astype(np.float64)) >= 0) or np.all(k[1:] >= k[:-1])
    pr = O.project(osc, cams[0], np.arange(osc.n_total))
    rect = pr["rect"][pr["visible"]]
    expect = ((rect[:, 2] - rect[:, 0] + 1) * (rect[:, 3] - rect[:, 1] + 1)).sum()
    assert expect == k.size
    # depth bits in the key are the FP32 depth of that Gaussian
    zb = (k & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
    assert np.array_equal(zb, pr["z"][g])


@pytest.mark.parametrize("k", [1, 2, 3])
def test_bin_lists_filtered_per_tile_give_tile_order(plain, k):
    """Key lists per bin of 2^k x 2^k tiles, built as the library builds them
    (a stable sort of the visible Gaussians, in index order, by their FP32
    depth bits, then a stable partition by every bin the tile rect >> k
    touches), filtered per tile by the tile rect, reproduce each tile's list
    of the key spec (tile, then depth bits, then index) and nothing else."""
    scene, cams, osc = plain
    cam = cams[0]
    gids = np.arange(osc.n_total)
    k_ref, g_ref = O.keys(osc, cam, gids)
    pr = O.project(osc, cam, gids)
    vis = np.flatnonzero(pr["visible"])
    zbits = pr["z"][vis].astype(np.float32).view(np.uint32)
    order = vis[np.argsort(zbits, kind="stable")]
    rect = pr["rect"]   # tile rect (tx0, ty0, tx1, ty1), inclusive
    bins = {}
    for r in order:
        x0, y0, x1, y1 = (int(v) >> k for v in rect[r])
        for by in range(y0, y1 + 1):
            for bx in range(x0, x1 + 1):
                bins.setdefault((bx, by), []).append(r)
    tiles_x = (cam.width + 15) // 16
    tiles_y = (cam.height + 15) // 16
    ref_tile = (k_ref >> np.uint64(32)).astype(np.int64)
    n_seen = 0
    for t in range(tiles_x * tiles_y):
        tx, ty = t % tiles_x, t // tiles_x
        lst = [r for r in bins.get((tx >> k, ty >> k), [])
               if rect[r, 0] <= tx <= rect[r, 2] and rect[r, 1] <= ty <= rect[r, 3]]
        assert np.array_equal(np.asarray(lst, np.int64), g_ref[ref_tile == t]), (k, t)
        n_seen += len(lst)
    assert n_seen == k_ref.size > 0


# --------------------------------------------------------------------------
# EWA projection and SH: textbook checks
# --------------------------------------------------------------------------
def test_ewa_matches_monte_carlo_projection():
    """For a small, distant Gaussian the projected covariance (minus the
    0.3 px^2 dilation) matches the sample covariance of perspective-projected
    3D samples (first-order EWA is exact in the small-Gaussian limit)."""
    rng = np.random.default_rng(11)
    q = rng.normal(size=4)
    sc = _single_level_scene([[0.3, -0.2, 4.0]], [np.log([0.02, 0.006, 0.012])], [q],
                             [0.0], [_sh_for_rgb((1, 1, 1))])
    cam = synth.look_at((0.1, 0.1, -3.0), (0.02, -0.03, 1.0), (0, -1, 0), 512, 512, 40.0)
    osc = O.OracleScene(sc)
    pr = O.project(osc, cam, np.arange(1))
    s = osc.scales[0].astype(np.float64)
    w, x, y, z = osc.quats[0].astype(np.float64)
    Rq = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                   [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                   [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    pts = rng.standard_normal((400_000, 3)) * s @ Rq.T + osc.means[0]
    Rc = cam.R.astype(np.float64); tc = cam.t.astype(np.float64)
    pc = pts @ Rc.T + tc
    u = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
    v = cam.fy * pc[:, 1] / pc[:, 2] + cam.cy
    cov = np.cov(np.stack([u, v]))
    got = np.array([[pr["cov"][0, 0] - 0.3, pr["cov"][0, 1]], [pr["cov"][0, 1], pr["cov"][0, 2] - 0.3]])
    assert np.allclose(got, cov, rtol=0.02, atol=0.02 * np.abs(cov).max())
    assert abs(pr["mean2"][0, 0] - u.mean()) < 0.05 and abs(pr["mean2"][0, 1] - v.mean()) < 0.05
    # conic is the inverse of the covariance
    C2 = np.array([[pr["cov"][0, 0], pr["cov"][0, 1]], [pr["cov"][0, 1], pr["cov"][0, 2]]])
    K = np.array([[pr["conic"][0, 0], pr["conic"][0, 1]], [pr["conic"][0, 1], pr["conic"][0, 2]]])
    assert np.allclose(C2 @ K, np.eye(2), atol=1e-12)


def _extent_q(o32):
    """Q of the key rect for an FP32 opacity: 2 ln(255 o_hi) * 1.001 with o_hi
    the upper end of o's bucket (FP32 exponent and three leading mantissa
    bits), restated from that definition."""
    bits = int(np.float32(o32).view(np.uint32))
    top = bits >> 20
    hi_bits = ((top + 1) << 20) if top <= (127 << 3) else ((127 << 3) + 1) << 20
    hi = float(np.uint32(hi_bits).view(np.float32))
    return float(np.float32(2.0 * math.log(255.0 * hi) * 1.001))


def test_jacobian_lateral_clamp_closed_form():
    """The EWA Jacobian is evaluated at x/z, y/z clamped to +-1.3 tan(fov/2)
    (tan(fovx/2) = W / (2 fx); 3DGS's rasteriser): for an isotropic Gaussian of
    std s at camera point (x, y, z) with R = I, Sigma' = (s f / z)^2 [[1 +
    uc^2, uc wc], [uc wc, 1 + wc^2]] + 0.3 I, uc, wc the clamped x/z, y/z,
    while the mean keeps the unclamped point.  Checked inside the limits (no
    change), past one limit and past both with negative signs; the FP32 key
    rect of each is the tile range of that covariance's extent."""
    cam = synth.plain_camera(256, 256)
    f = float(cam.fx)
    lim = float(np.float32(1.3 * (256 / (2.0 * f))))
    assert abs(lim - 1.3 * math.tan(math.radians(30.0))) < 1e-6
    sigma, o = 0.5, 0.8
    pts = [(1.5, 0.0), (3.0, 0.9), (-3.3, -3.6)]          # camera (x, y) at z = 3
    sc = _single_level_scene([[x, y, 0.0] for x, y in pts], [[math.log(sigma)] * 3] * 3,
                             [[1, 0, 0, 0]] * 3, [_logit(o)] * 3, [_sh_for_rgb((1, 1, 1))] * 3)
    osc = O.OracleScene(sc)
    pr = O.project(osc, cam, np.arange(3))
    assert pr["visible"].all()
    se = float(osc.scales[0, 0])
    k = (se * f / 3.0) ** 2
    o32 = float(pr["o32"][0])
    Q = _extent_q(o32)
    for i, (x, y) in enumerate(pts):
        u, w = float(np.float32(x)) / 3.0, float(np.float32(y)) / 3.0   # stored in FP32
        uc, wc = min(max(u, -lim), lim), min(max(w, -lim), lim)
        expect = np.array([k * (1 + uc * uc) + 0.3, k * uc * wc, k * (1 + wc * wc) + 0.3])
        assert np.allclose(pr["cov"][i], expect, rtol=1e-9, atol=1e-9), (i, pr["cov"][i], expect)
        assert abs(pr["mean2"][i, 0] - (f * u + cam.cx)) < 1e-9
        assert abs(pr["mean2"][i, 1] - (f * w + cam.cy)) < 1e-9
        plain = np.array([k * (1 + u * u) + 0.3, k * u * w, k * (1 + w * w) + 0.3])
        assert (i == 0) == np.allclose(plain, expect), i
        # key rect: pixel range [ceil(m - r - 0.5), floor(m + r - 0.5)],
        # r = sqrt(Q Sigma'_kk), clipped to the image, in tiles of 16
        mx, my = f * u + cam.cx, f * w + cam.cy
        rx, ry = math.sqrt(Q * expect[0]), math.sqrt(Q * expect[2])
        x0 = max(math.ceil(mx - rx - 0.5), 0); x1 = min(math.floor(mx + rx - 0.5), 255)
        y0 = max(math.ceil(my - ry - 0.5), 0); y1 = min(math.floor(my + ry - 0.5), 255)
        assert tuple(pr["rect"][i]) == (x0 // 16, y0 // 16, x1 // 16, y1 // 16), (i, pr["rect"][i])


def test_quaternion_normalisation():
    """Activation's unit quaternion: for raw q of any scale the output has unit
    norm to FP32 rounding and is parallel to q (q_i |q^| = q^_i |q|); and a
    Gaussian whose raw quaternion is k (cos th/2, sin th/2 a) for k far from 1
    projects to J (Rod(a, th) diag(s^2) Rod^T) J^T + 0.3 I, with the rotation
    built by Rodrigues' formula from the axis and angle, not from the oracle's
    quaternion."""
    rng = np.random.default_rng(21)
    n = 64
    scale = 10.0 ** rng.uniform(-6, 6, n)
    q = (rng.normal(size=(n, 4)) * scale[:, None]).astype(np.float32)
    _, qn, _ = O.activate(np.zeros((n, 3), np.float32), q, np.zeros(n, np.float32))
    qd = q.astype(np.float64); qnd = qn.astype(np.float64)
    assert np.abs(np.linalg.norm(qnd, axis=1) - 1).max() < 4 * 2.0 ** -24
    qu = qd / np.linalg.norm(qd, axis=1, keepdims=True)
    assert np.abs(qnd - qu).max() < 2.0 ** -24
    # projection of a rotated anisotropic Gaussian at the image centre
    cam = synth.plain_camera(64, 64)
    s = np.array([0.03, 0.011, 0.02])
    for k, (ax, th) in zip([7.25, 1e-3, 3e4], [((1, 2, 3), 0.7), ((-2, 0.5, 1), 2.1), ((0, 0, 1), -1.2)]):
        a = np.asarray(ax, np.float64); a /= np.linalg.norm(a)
        qr = k * np.array([math.cos(th / 2), *(math.sin(th / 2) * a)])
        sc = _single_level_scene([[0, 0, 0]], [np.log(s)], [qr], [0.0], [_sh_for_rgb((1, 1, 1))])
        osc = O.OracleScene(sc)
        pr = O.project(osc, cam, np.arange(1))
        Kx = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
        Rod = np.eye(3) + math.sin(th) * Kx + (1 - math.cos(th)) * Kx @ Kx
        se = osc.scales[0].astype(np.float64)
        Sig = Rod @ np.diag(se ** 2) @ Rod.T
        f = cam.fx / 3.0
        expect = f * f * Sig[:2, :2] + 0.3 * np.eye(2)
        got = np.array([[pr["cov"][0, 0], pr["cov"][0, 1]], [pr["cov"][0, 1], pr["cov"][0, 2]]])
        assert np.allclose(got, expect, rtol=1e-6, atol=1e-6 * np.abs(expect).max()), (k, got, expect)


def test_sh_basis_orthonormal():
    """The 16 real SH functions are orthonormal on the sphere (Gauss-Legendre
    in cos(theta) x uniform phi quadrature, exact for these degrees)."""
    xg, wg = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phis = np.arange(nphi) * 2 * np.pi / nphi
    G = np.zeros((16, 16))
    for ct, w in zip(xg, wg):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            Y = O.sh_basis((st * math.cos(ph), st * math.sin(ph), ct))
            G += np.outer(Y, Y) * w * (2 * np.pi / nphi)
    assert np.allclose(G, np.eye(16), atol=1e-12)


def test_sh_degree0_constant_colour():
    rng = np.random.default_rng(5)
    n = 50
    sh = np.zeros((n, 16, 3), np.float32)
    sh[:, 0, :] = rng.normal(0, 0.5, (n, 3))
    sc = _single_level_scene(rng.uniform(-1, 1, (n, 3)), np.full((n, 3), -3.0),
                             rng.normal(size=(n, 4)), np.zeros(n), sh)
    osc = O.OracleScene(sc)
    pr = O.project(osc, synth.plain_camera(), np.arange(n))
    y00 = 0.5 / math.sqrt(math.pi)
    expect = np.maximum(0, sh[:, 0, :].astype(np.float64) * y00 + 0.5)
    v = pr["visible"]
    assert np.abs(pr["rgb"][v] - expect[v]).max() < 1e-12


def test_sh_direction_dependence():
    """Degree-1 coefficient on the y basis: colour = Y1,-1(dir) k + 0.5, with
    dir the unit vector from the camera centre to the mean."""
    sh = np.zeros((1, 16, 3), np.float32)
    sh[0, 1, :] = 0.7
    sc = _single_level_scene([[0.5, 0.3, 0.0]], [[-3.0] * 3], [[1, 0, 0, 0]], [0.0], sh)
    cam = synth.plain_camera()
    pr = O.project(O.OracleScene(sc), cam, np.arange(1))
    d = np.array([0.5, 0.3, 0.0], np.float32).astype(np.float64) - cam.center
    d /= np.linalg.norm(d)
    k = float(np.float32(0.7))
    expect = k * math.sqrt(3 / (4 * math.pi)) * d[1] + 0.5
    assert abs(pr["rgb"][0, 0] - expect) < 1e-12


def test_filter_opacity_compensation():
    """Eq. 3: the 3D filter adds v to the covariance and scales the opacity by
    sqrt(|Sigma| / |Sigma + v I|) = prod_k s_k / sqrt(s_k^2 + v)."""
    s = np.array([0.05, 0.02, 0.03])
    v = 0.01 ** 2
    sc = _single_level_scene([[0, 0, 0]], [np.log(s)], [[1, 0, 0, 0]], [0.0],
                             [_sh_for_rgb((1, 1, 1))], filter_var=v)
    sc0 = _single_level_scene([[0, 0, 0]], [np.log(np.sqrt(s ** 2 + v))], [[1, 0, 0, 0]], [0.0],
                              [_sh_for_rgb((1, 1, 1))])
    cam = synth.plain_camera()
    p1 = O.project(O.OracleScene(sc), cam, np.arange(1))
    p0 = O.project(O.OracleScene(sc0), cam, np.arange(1))
    osc = O.OracleScene(sc)
    sf = osc.scales[0].astype(np.float64)
    comp = np.prod(sf / np.sqrt(sf ** 2 + v))
    assert abs(p1["opacity"][0] - 0.5 * comp) < 1e-7
    assert np.allclose(p1["cov"], p0["cov"], rtol=1e-5)


# --------------------------------------------------------------------------
# Eq. 2 active sets
# --------------------------------------------------------------------------
def _small_outdoor(scale=0.004, seed=1):
    side = 1000.0 * math.sqrt(scale)
    return synth.outdoor_scene(seed=seed, n0=int(16_000_000 * scale), num_levels=4,
                               extent=side, grid=2)


def test_lod_partition_of_identical_levels():
    """If every level holds the same means, each position is selected at
    exactly one level (the distance bands of Eq. 2 partition [0, inf))."""
    sc = _small_outdoor()
    base = sc.levels[0]
    lv = [synth.Level(base.means, base.log_scales, base.quats, base.opacity_logits, base.sh)
          for _ in range(4)]
    sc2 = synth.Scene(levels=lv, d_thresholds=np.array([10.0, 20.0, 40.0]),
                      chunk_centers=sc.chunk_centers)
    osc = O.OracleScene(sc2)
    c = np.array([sc.extent / 2, sc.extent / 2, 3.0])
    g, _ = O.lod_select(osc, c)
    n = base.n
    counts = np.bincount(g % n, minlength=n)
    assert np.all(counts == 1)
    # and the level chosen matches the distance band computed here in FP64
    lvl = g // n
    d = np.linalg.norm(base.means[g % n].astype(np.float64) - c, axis=1)
    band = np.searchsorted(np.array([10.0, 20.0, 40.0]), d, side="right")
    assert (lvl != band).sum() <= 2


def test_lod_single_level_and_infinite_threshold_is_full():
    sc = _small_outdoor()
    osc = O.OracleScene(sc)
    c = sc.chunk_centers[0]
    g, _ = O.lod_select(osc, c, d_inner=[np.inf, np.inf, np.inf])
    assert np.array_equal(g, np.arange(osc.level_off[1]))


def test_lod_select_brute_numpy():
    """Eq. 2 written out with numpy in FP64 agrees except on Gaussians within
    FP32 rounding of a threshold sphere; the oracle counts those."""
    sc = _small_outdoor()
    osc = O.OracleScene(sc)
    c = np.array([30.0, 40.0, 5.0])
    g, dis = O.lod_select(osc, c)
    sel = np.zeros(osc.n_total, bool)
    d = np.array([0.0, 10.0, 20.0, 40.0, np.inf])
    for l in range(4):
        a, b = osc.level_off[l], osc.level_off[l + 1]
        r = np.linalg.norm(osc.means[a:b].astype(np.float64) - c, axis=1)
        sel[a:b] = (d[l] <= r) & (r < d[l + 1])
    mine = np.zeros(osc.n_total, bool); mine[g] = True
    assert (mine != sel).sum() == dis
    assert dis <= 3


def test_chunk_radius_grid():
    c = np.array([[62.5 * (i + 0.5), 62.5 * (j + 0.5), 2.0] for j in range(4) for i in range(4)])
    assert np.allclose(O.chunk_radius(c), 62.5)
    assert O.chunk_radius(c[:1])[0] == 0.0


def test_single_chunk_radius_zero_equals_lod_at_centre():
    sc = _small_outdoor()
    sc1 = synth.Scene(levels=sc.levels, d_thresholds=sc.d_thresholds,
                      chunk_centers=sc.chunk_centers[:1].copy())
    osc = O.OracleScene(sc1)
    a = O.chunk_select(osc, 0)
    b, _ = O.lod_select(osc, sc1.chunk_centers[0])
    assert np.array_equal(a, b)


def test_chunk_select_offsets_thresholds_by_radius():
    sc = _small_outdoor()
    osc = O.OracleScene(sc)
    r = O.chunk_radius(osc.centers)
    for k in range(osc.centers.shape[0]):
        a = O.chunk_select(osc, k)
        b, _ = O.lod_select(osc, osc.centers[k], d_inner=osc.d_inner + r[k])
        assert np.array_equal(a, b)


# --------------------------------------------------------------------------
# Eq. 4 chunk choice and opacity blending
# --------------------------------------------------------------------------
def test_chunk_weights_sum_to_one_unclamped():
    rng = np.random.default_rng(2)
    for _ in range(100):
        mA, mB, c = rng.normal(size=(3, 3)) * 10
        assert abs(O.chunk_tsum_unclamped(mA, mB, c) - 1.0) < 1e-12


def test_chunk_pick_closed_form():
    cen = np.array([[0, 0, 0], [10, 0, 0], [0, 10, 0], [10, 10, 0]], np.float64)
    A, B, tA, tB = O.chunk_pick(cen, [2.0, 1.0, 0.0])
    assert (A, B) == (0, 1)
    assert abs(tA - 0.8) < 1e-12 and abs(tB - 0.2) < 1e-12
    A, B, tA, tB = O.chunk_pick(cen, [0.0, 0.0, 0.0])
    assert (A, tA, tB) == (0, 1.0, 0.0)
    # beyond the far centre's projection: clamped
    A, B, tA, tB = O.chunk_pick(cen, [-3.0, 0.5, 0.0])
    assert (A, B) == (0, 2) and abs(tA - 0.95) < 1e-12 and abs(tB - 0.05) < 1e-12
    A, B, tA, tB = O.chunk_pick(cen[:2], [-3.0, 0.5, 0.0])  # unclamped 1.3 / -0.3
    assert (A, B) == (0, 1) and tA == 1.0 and tB == 0.0
    # equidistant: lower index wins
    A, B, _, _ = O.chunk_pick(cen, [5.0, 5.0, 0.0])
    assert (A, B) == (0, 1)
    A, B, tA, tB = O.chunk_pick(cen[:1], [3.0, 0, 0])
    assert B == -1 and tA == 1.0


def test_chunk_union_multipliers():
    a = np.array([1, 3, 5, 7]); b = np.array([2, 3, 6, 7, 9])
    g, m = O.chunk_union(a, b, 0.25, 0.75)
    assert list(g) == [1, 2, 3, 5, 6, 7, 9]
    assert list(m) == [0.25, 0.75, 1.0, 0.25, 0.75, 1.0, 0.75]


@pytest.fixture(scope="module")
def small_outdoor_osc():
    sc = _small_outdoor(scale=0.01, seed=3)
    return sc, O.OracleScene(sc)


def test_blend_at_chunk_centre_equals_chunk_alone(small_outdoor_osc):
    """Camera exactly at m_A: t_B = 0, so B-only Gaussians vanish and the
    blended render equals the render of chunk A's set alone."""
    sc, osc = small_outdoor_osc
    mA = sc.chunk_centers[0]
    cam = synth.look_at(mA, (1.0, 0.3, -0.15), (0, 0, 1), 96, 64, 70.0)
    gb, mb, info = O.active_set(osc, O.MODE_CHUNK_BLEND, cam)
    assert info["A"] == 0 and info["tB"] == 0.0
    ga, _, _ = O.active_set(osc, O.MODE_CHUNK, cam)
    r1 = O.render(osc, cam, gb, mb)
    r2 = O.render(osc, cam, ga)
    assert np.array_equal(r1["rgb"], r2["rgb"])


def test_blend_continuous_across_midpoint(small_outdoor_osc):
    """Crossing the bisector swaps A and B but t_A = t_B = 1/2 on it, so the
    image is continuous (small camera step gives a small image change)."""
    sc, osc = small_outdoor_osc
    m0, m1 = sc.chunk_centers[0], sc.chunk_centers[1]
    mid = 0.5 * (m0 + m1)
    dirn = (m1 - m0) / np.linalg.norm(m1 - m0)
    imgs = []
    for eps in (-1e-6, 1e-6):
        cam = synth.look_at(mid + eps * dirn, (0.2, 1.0, -0.15), (0, 0, 1), 96, 64, 70.0)
        g, m, info = O.active_set(osc, O.MODE_CHUNK_BLEND, cam)
        imgs.append((info["A"], O.render(osc, cam, g, m)["rgb"]))
    assert imgs[0][0] != imgs[1][0]
    assert np.abs(imgs[0][1] - imgs[1][1]).max() < 1e-4


def test_intersection_never_modulated(small_outdoor_osc):
    sc, osc = small_outdoor_osc
    a, b = O.chunk_select(osc, 0), O.chunk_select(osc, 1)
    g, m = O.chunk_union(a, b, 0.3, 0.7)
    both = np.isin(g, np.intersect1d(a, b))
    assert np.all(m[both] == 1.0)
    assert np.all(m[~both & np.isin(g, a)] == np.float32(0.3))
    assert np.all(m[~both & np.isin(g, b)] == np.float32(0.7))
