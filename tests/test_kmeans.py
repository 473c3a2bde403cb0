"""Chunk centres from camera positions (supplementary "Selecting chunk
centers", Eq. 5): the oracle pinned to closed forms and fixed-point
properties of K-means, and the library's host implementation (through the
C ABI; it needs no device) equal to the oracle bit for bit."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2505_23158_gb300 import synth


def test_num_clusters_closed_form():
    # positions on a circle of radius R (mean at its centre): N = ceil(4R/d1)
    R, d1 = 37.0, 10.0
    ang = np.linspace(0, 2 * math.pi, 64, endpoint=False)
    p = np.stack([R * np.cos(ang) + 5, R * np.sin(ang) - 3, np.full(64, 2.0)], 1)
    assert O.num_clusters(p, d1) == math.ceil(4 * R / d1) == 15
    assert O.num_clusters(p[:1], d1) == 1                # a single camera
    assert O.num_clusters(p[:8], 0.01) == 8              # clamped to the camera count


def test_kmeans_separated_blobs():
    rng = np.random.default_rng(0)
    centres = np.array([[0, 0, 0], [100, 0, 0], [0, 100, 5]], np.float64)
    labels = np.repeat(np.arange(3), 20)
    p = centres[labels] + rng.normal(scale=1.0, size=(60, 3))
    m, a, it = O.kmeans_centers(p, [0, 20, 40])
    assert np.array_equal(a, labels)
    for j in range(3):
        assert np.allclose(m[j], p[labels == j].mean(0), atol=1e-12)
    assert it >= 1


def test_kmeans_fixed_point_and_monotone():
    cams = synth.outdoor_trajectory(synth.outdoor_scene(seed=1, n0=1000, num_levels=1),
                                    seed=1, n_poses=200)
    p = synth.camera_positions(cams)
    k = 12
    init = synth.kmeans_init(len(p), k, seed=2)
    m, a, it = O.kmeans_centers(p, init, max_iter=200)
    assert it < 200                                      # converged
    for j in range(k):
        if (a == j).any():
            assert np.allclose(m[j], p[a == j].mean(0), atol=1e-9)
    d = ((p[:, None, :] - m[None]) ** 2).sum(-1)
    assert np.array_equal(a, d.argmin(1))
    obj = []
    for n_it in range(1, 6):
        mm, aa, _ = O.kmeans_centers(p, init, max_iter=n_it)
        obj.append(((p - mm[aa]) ** 2).sum())
    assert all(b <= a0 + 1e-9 for a0, b in zip(obj, obj[1:]))


@pytest.mark.gpu
def test_library_matches_oracle():
    pytest.importorskip("torch")
    from paper_2505_23158_gb300 import api, build
    build.build()
    cams = synth.outdoor_trajectory(synth.outdoor_scene(seed=3, n0=1000, num_levels=1),
                                    seed=3, n_poses=300)
    p = synth.camera_positions(cams)
    k = O.num_clusters(p, 10.0)
    assert api.num_clusters(p, 10.0) == k
    init = synth.kmeans_init(len(p), k, seed=4)
    for max_iter in (0, 1, 3, 100):
        m_ref, a_ref, it_ref = O.kmeans_centers(p, init, max_iter=max_iter)
        m, a, it = api.kmeans_centers(p, init, max_iter=max_iter)
        assert it == it_ref
        assert np.array_equal(m, m_ref)                  # bit for bit
        assert np.array_equal(a, a_ref)
