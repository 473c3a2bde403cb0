"""Scene files and level checkpoints.

A scene file holds everything `Lodge.load_scene` needs, so a scene built (or
fine-tuned) once can be reloaded without regenerating it:
  * per level, the raw parameters in the library's layout (means, log-scales,
    quaternions, opacity logits, SH (N, 16, 3)) and the Eq. 3 filter variance;
  * the depth thresholds d_1 .. d_{L-1}, the chunk centres, the SH degree,
    the 2D-filter flag, the world extent and the heightfield parameters.
It is one uncompressed `.npz` archive (numpy's format: a zip of `.npy`
arrays), so a scene of N Gaussians takes about 236 N bytes plus a few KB.

A level checkpoint is the five parameter tensors of one level (for instance
G_l after `lod_build.build_level`), saved with `torch.save` on the host.
"""
from __future__ import annotations

import json
from typing import Sequence

import numpy as np

from . import synth

FORMAT_VERSION = 1
_FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def save_scene(path: str, scene: synth.Scene) -> None:
    """Write `scene` to `path` (an .npz archive)."""
    arrays = {}
    meta = {"version": FORMAT_VERSION, "num_levels": scene.num_levels, "sh_degree": int(scene.sh_degree),
            "filter2d": bool(scene.filter2d), "extent": float(scene.extent),
            "filter_var": [float(l.filter_var) for l in scene.levels],
            "height_params": None}
    for i, lv in enumerate(scene.levels):
        for f in _FIELDS:
            arrays[f"level{i}_{f}"] = np.ascontiguousarray(getattr(lv, f), np.float32)
    arrays["d_thresholds"] = np.asarray(scene.d_thresholds, np.float64)
    arrays["chunk_centers"] = np.asarray(scene.chunk_centers, np.float64)
    if scene.height_params is not None:
        meta["height_params"] = sorted(scene.height_params)
        for k, v in scene.height_params.items():
            arrays[f"height_{k}"] = np.asarray(v, np.float64)
    arrays["meta"] = np.frombuffer(json.dumps(meta).encode(), np.uint8)
    with open(path, "wb") as fh:
        np.savez(fh, **arrays)


def load_scene(path: str) -> synth.Scene:
    """Read a scene written by `save_scene`."""
    with np.load(path, allow_pickle=False) as z:
        meta = json.loads(bytes(z["meta"]).decode())
        if meta.get("version") != FORMAT_VERSION:
            raise ValueError(f"{path}: scene file version {meta.get('version')}, expected {FORMAT_VERSION}")
        levels = []
        for i in range(meta["num_levels"]):
            a = {f: z[f"level{i}_{f}"] for f in _FIELDS}
            n = a["means"].shape[0]
            if (a["log_scales"].shape != (n, 3) or a["quats"].shape != (n, 4)
                    or a["opacity_logits"].shape != (n,) or a["sh"].shape != (n, synth.SH_COEFFS, 3)):
                raise ValueError(f"{path}: level {i} has inconsistent array shapes")
            levels.append(synth.Level(a["means"], a["log_scales"], a["quats"], a["opacity_logits"], a["sh"],
                                      float(meta["filter_var"][i])))
        hp = None
        if meta["height_params"] is not None:
            hp = {k: z[f"height_{k}"] for k in meta["height_params"]}
        return synth.Scene(levels=levels, d_thresholds=z["d_thresholds"], chunk_centers=z["chunk_centers"],
                           sh_degree=int(meta["sh_degree"]), extent=float(meta["extent"]), height_params=hp,
                           filter2d=bool(meta["filter2d"]))


def save_level(path: str, params: Sequence) -> None:
    """Save one level's five parameter tensors (means, log_scales, quats,
    logits, sh (N, 48)) on the host."""
    import torch
    if len(params) != 5:
        raise ValueError("a level has five parameter tensors")
    torch.save({"version": FORMAT_VERSION, "params": [t.detach().cpu() for t in params]}, path)


def load_level(path: str, device=None) -> tuple:
    """Load a level saved by `save_level`, optionally onto `device`."""
    import torch
    d = torch.load(path, map_location="cpu")
    if d.get("version") != FORMAT_VERSION or len(d.get("params", ())) != 5:
        raise ValueError(f"{path}: not a level checkpoint of version {FORMAT_VERSION}")
    ps = d["params"]
    return tuple(p.to(device) if device is not None else p for p in ps)


def level_of_params(params: Sequence, filter_var: float = 0.0) -> synth.Level:
    """A synth.Level (host arrays) from one level's parameter tensors, for
    building a scene file from a fine-tuned level."""
    m, ls, q, lg, sh = [np.ascontiguousarray(t.detach().cpu().numpy(), np.float32) for t in params]
    return synth.Level(m, ls, q, lg, sh.reshape(m.shape[0], synth.SH_COEFFS, 3), float(filter_var))
