"""The build loop's SSIM (CPU): identical images give 1, and the value
equals a brute-force evaluation of the definition (local Gaussian-window
means, variances and covariance with zero padding, C1 = 0.01^2,
C2 = 0.03^2) on small images."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _ssim_brute(a, b, size=11, sigma=1.5):
    H, W, C = a.shape
    r = size // 2
    g = np.array([math.exp(-(i - r) ** 2 / (2 * sigma * sigma)) for i in range(size)])
    g /= g.sum()
    w = np.outer(g, g)
    tot = 0.0
    for c in range(C):
        x = np.pad(a[..., c], r)
        y = np.pad(b[..., c], r)
        for i in range(H):
            for j in range(W):
                px = x[i:i + size, j:j + size]
                py = y[i:i + size, j:j + size]
                mx, my = (w * px).sum(), (w * py).sum()
                sxx = (w * px * px).sum() - mx * mx
                syy = (w * py * py).sum() - my * my
                sxy = (w * px * py).sum() - mx * my
                c1, c2 = 0.01 ** 2, 0.03 ** 2
                tot += ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return tot / (H * W * C)


def test_ssim_matches_definition():
    from paper_2505_23158_gb300 import lod_build
    rng = np.random.default_rng(3)
    a = rng.uniform(0, 1, (13, 17, 3))
    b = np.clip(a + rng.normal(0, 0.1, a.shape), 0, 1)
    got = float(lod_build.ssim(torch.tensor(a, dtype=torch.float64).float(),
                               torch.tensor(b, dtype=torch.float64).float()))
    assert abs(got - _ssim_brute(a, b)) < 1e-4
    same = float(lod_build.ssim(torch.tensor(a).float(), torch.tensor(a).float()))
    assert abs(same - 1.0) < 1e-5
    l = lod_build.dssim_l1(torch.tensor(a).float(), torch.tensor(b).float(), 0.2)
    l1 = float(np.abs(a - b).mean())
    assert abs(float(l) - (0.8 * l1 + 0.2 * (1 - got))) < 1e-4
    assert float(lod_build.dssim_l1(torch.tensor(a).float(), torch.tensor(b).float(), 0.0)) == pytest.approx(l1, abs=1e-6)
