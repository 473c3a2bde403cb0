"""Scene files and level checkpoints round-trip exactly (CPU)."""
import numpy as np
import pytest

import oracle as O
from paper_2505_23158_gb300 import scene_io, synth


def test_scene_file_round_trip(tmp_path):
    scene, cams = synth.workload_outdoor(seed=4, n_poses=3, scale=0.002, width=64, height_px=48)
    scene.levels[1].filter_var = 0.0123
    p = tmp_path / "scene.npz"
    scene_io.save_scene(str(p), scene)
    back = scene_io.load_scene(str(p))
    assert back.num_levels == scene.num_levels and back.sh_degree == scene.sh_degree
    assert back.filter2d == scene.filter2d and back.extent == scene.extent
    assert np.array_equal(back.d_thresholds, scene.d_thresholds)
    assert np.array_equal(back.chunk_centers, scene.chunk_centers)
    for a, b in zip(scene.levels, back.levels):
        for f in ("means", "log_scales", "quats", "opacity_logits", "sh"):
            assert np.array_equal(getattr(a, f), getattr(b, f)), f
        assert a.filter_var == b.filter_var
    for k in scene.height_params:
        assert np.array_equal(scene.height_params[k], back.height_params[k])
    # the reloaded scene renders identically (oracle)
    cam = cams[1]
    g, m, _ = O.active_set(O.OracleScene(scene), O.MODE_CHUNK_BLEND, cam)
    g2, m2, _ = O.active_set(O.OracleScene(back), O.MODE_CHUNK_BLEND, cam)
    assert np.array_equal(g, g2)
    r1 = O.render(O.OracleScene(scene), cam, g, m, bounds=False)
    r2 = O.render(O.OracleScene(back), cam, g2, m2, bounds=False)
    assert np.array_equal(r1["rgb"], r2["rgb"])


def test_level_checkpoint_round_trip(tmp_path):
    torch = pytest.importorskip("torch")
    lv = synth.plain_scene(2, n=100).levels[0]
    params = [torch.from_numpy(np.ascontiguousarray(a, np.float32)) for a in
              (lv.means, lv.log_scales, lv.quats, lv.opacity_logits, lv.sh.reshape(100, 48))]
    p = tmp_path / "level.pt"
    scene_io.save_level(str(p), params)
    back = scene_io.load_level(str(p))
    assert all(torch.equal(a, b) for a, b in zip(params, back))
    lv2 = scene_io.level_of_params(back, 0.5)
    assert np.array_equal(lv2.sh, lv.sh) and lv2.filter_var == 0.5


def test_scene_file_rejects_other_versions(tmp_path):
    scene = synth.plain_scene(0, n=10)
    p = tmp_path / "s.npz"
    scene_io.save_scene(str(p), scene)
    with np.load(str(p)) as z:
        arrays = dict(z)
    import json
    meta = json.loads(bytes(arrays["meta"]).decode())
    meta["version"] = 99
    arrays["meta"] = np.frombuffer(json.dumps(meta).encode(), np.uint8)
    with open(str(p), "wb") as fh:
        np.savez(fh, **arrays)
    with pytest.raises(ValueError):
        scene_io.load_scene(str(p))
