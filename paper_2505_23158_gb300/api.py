"""Python face of the C ABI: device memory and streams come from PyTorch,
every step of the render runs in liblodge.so.

    ctx = Lodge(device=0)
    sid = ctx.load_scene(scene)                    # synth.Scene (host arrays)
    img, stats = ctx.render(sid, CHUNK_BLEND, cam) # cuda float32 (H, W, 3)
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _capi as A
from ._capi import CHUNK, CHUNK_BLEND, FULL, LOD, RESIDENT, STREAMED, LodgeError  # noqa: F401


def camera_struct(cam) -> A.lodge_camera:
    c = A.lodge_camera()
    c.R[:] = [float(x) for x in np.asarray(cam.R, np.float32).ravel()]
    c.t[:] = [float(x) for x in np.asarray(cam.t, np.float32).ravel()]
    c.fx, c.fy = float(np.float32(cam.fx)), float(np.float32(cam.fy))
    c.cx, c.cy = float(np.float32(cam.cx)), float(np.float32(cam.cy))
    c.width, c.height = int(cam.width), int(cam.height)
    c.znear = float(np.float32(cam.znear))
    c.center[:] = [float(x) for x in np.asarray(cam.center, np.float64)]
    return c


def camera_array(cams) -> C.Array:
    arr = (A.lodge_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = camera_struct(c)
    return arr


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def stats_dict(s: A.lodge_frame_stats) -> dict:
    return dict(n_active=s.n_active, n_visible=s.n_visible, n_keys=s.n_keys, n_tiles=s.n_tiles,
                chunk_a=s.chunk_a, chunk_b=s.chunk_b, t_a=s.t_a, t_b=s.t_b)


class Lodge:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.device = int(device)
        h = C.c_void_p()
        A.call("lodge_create", self.device, int(hbm_budget_bytes), C.byref(h))
        self._h = h
        self._keep = {}
        self._num_levels = {}
        self._n_total = {}

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            A.call("lodge_destroy", self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- scenes
    def load_scene(self, scene, residency: int = 0) -> int:
        """Copy a synth.Scene into the library.  residency=STREAMED keeps the
        levels in pinned host memory and gathers chunk blocks into HBM on use."""
        levels = (A.lodge_level_desc * scene.num_levels)()
        keep = []
        for i, lv in enumerate(scene.levels):
            arrs = [np.ascontiguousarray(a, np.float32) for a in
                    (lv.means, lv.log_scales, lv.quats, lv.opacity_logits, lv.sh)]
            keep += arrs
            levels[i].n = lv.n
            levels[i].means, levels[i].log_scales, levels[i].quats, levels[i].opacity_logits, \
                levels[i].sh = [a.ctypes.data for a in arrs]
            levels[i].filter_var = float(lv.filter_var)
        d = np.ascontiguousarray(scene.d_thresholds, np.float64)
        cc = np.ascontiguousarray(scene.chunk_centers, np.float64)
        desc = A.lodge_scene_desc()
        desc.num_levels = scene.num_levels
        desc.sh_degree = int(scene.sh_degree)
        desc.levels = C.cast(levels, C.c_void_p)
        desc.d_thresholds = d.ctypes.data if d.size else None
        desc.num_chunks = int(cc.shape[0])
        desc.chunk_centers = cc.ctypes.data if cc.size else None
        desc.residency = int(residency)
        desc.filter2d = int(bool(getattr(scene, "filter2d", False)))
        sid = C.c_int32()
        A.call("lodge_load_scene", self._h, C.byref(desc), C.byref(sid))
        self._num_levels[sid.value] = scene.num_levels
        self._n_total[sid.value] = scene.n_total
        return sid.value

    def unload_scene(self, sid: int):
        A.call("lodge_unload_scene", self._h, int(sid))

    def upload_chunks(self, sid: int, chunk_ids: Sequence[int], blocking: bool = True):
        ids = np.ascontiguousarray(chunk_ids, np.int32)
        A.call("lodge_upload_chunks", self._h, int(sid), ids.ctypes.data if ids.size else None,
               int(ids.size), int(blocking))

    # -- selection
    def select(self, sid: int, mode: int, cam, want_gids: bool = False, stream=None):
        """(selection dict, gids uint32 cuda tensor or None)."""
        sel = (A.lodge_selection * 1)()
        cams = camera_array([cam])
        gids = None
        if want_gids:
            A.call("lodge_select_lod", self._h, int(sid), int(mode), cams, 1, sel, None, 0,
                   _stream(stream))
            n = sel[0].n_active
            gids = torch.empty(max(n, 1), dtype=torch.int32, device=f"cuda:{self.device}")
            A.call("lodge_select_lod", self._h, int(sid), int(mode), cams, 1, sel,
                   _ptr(gids), n, _stream(stream))
            gids = gids[:n]
        else:
            A.call("lodge_select_lod", self._h, int(sid), int(mode), cams, 1, sel, None, 0,
                   _stream(stream))
        s = sel[0]
        return dict(chunk_a=s.chunk_a, chunk_b=s.chunk_b, t_a=s.t_a, t_b=s.t_b,
                    n_active=s.n_active), gids

    def select_thresholds(self, sid: int, views, candidates, stream=None):
        """Greedy depth-threshold search over the views: (d, keys) with d the
        num_levels - 1 chosen thresholds (inf where no candidate was left) and
        keys[l - 1, k] the tile keys of candidate k at step l (-1: not
        eligible)."""
        L = self._num_levels[sid]
        cand = np.ascontiguousarray(candidates, np.float64)
        d = np.zeros(max(L - 1, 1), np.float64)
        keys = np.zeros((max(L - 1, 1), cand.size), np.int64)
        vl = list(views)
        A.call("lodge_select_thresholds", self._h, int(sid), camera_array(vl), len(vl),
               C.c_void_p(cand.ctypes.data), int(cand.size), C.c_void_p(d.ctypes.data),
               C.c_void_p(keys.ctypes.data), _stream(stream))
        return d[:L - 1], keys[:L - 1]

    def render_lod(self, sid: int, cams, d_inner, stream=None):
        """LOD renders with per-camera thresholds (rows of num_levels - 1).
        Returns (images, stats)."""
        cl = list(cams)
        L = self._num_levels[sid]
        d = np.ascontiguousarray(d_inner, np.float64).reshape(len(cl), max(L - 1, 0))
        total = sum(c.width * c.height * 3 for c in cl)
        out = torch.empty(max(total, 1), dtype=torch.float32, device=f"cuda:{self.device}")
        st = (A.lodge_frame_stats * len(cl))()
        A.call("lodge_render_lod", self._h, int(sid), camera_array(cl), len(cl),
               C.c_void_p(d.ctypes.data) if d.size else None, _ptr(out), _stream(stream), st)
        imgs, off = [], 0
        for c in cl:
            n = c.width * c.height * 3
            imgs.append(out[off:off + n].view(c.height, c.width, 3))
            off += n
        return imgs, [stats_dict(s) for s in st]

    def importance(self, sid: int, mode: int, cams, score: Optional[torch.Tensor] = None,
                   chunk: int = -1, stream=None) -> torch.Tensor:
        """Largest blending weight per Gaussian over the cameras (float32
        cuda tensor of n_total, raised in place if given)."""
        cl = list(cams)
        if score is None:
            score = torch.zeros(self._n_total[sid], dtype=torch.float32,
                                device=f"cuda:{self.device}")
        A.call("lodge_importance", self._h, int(sid), int(mode), int(chunk), camera_array(cl),
               len(cl), _ptr(score), _stream(stream))
        return score

    def filter_chunk(self, sid: int, chunk: int, score: torch.Tensor, threshold: float,
                     stream=None) -> int:
        """Visibility filtering: drop chunk's Gaussians scoring below threshold;
        returns the new size of its set."""
        n = C.c_int64(0)
        A.call("lodge_filter_chunk", self._h, int(sid), int(chunk), _ptr(score),
               float(threshold), C.byref(n), _stream(stream))
        return n.value

    # -- render
    def render(self, sid: int, mode: int, cams, out: Optional[torch.Tensor] = None,
               stream=None, save: bool = False):
        """Render one camera (or a list).  Returns (image(s), stats list[, handle])."""
        single = not isinstance(cams, (list, tuple))
        cl = [cams] if single else list(cams)
        total = sum(c.width * c.height * 3 for c in cl)
        if out is None:
            out = torch.empty(total, dtype=torch.float32, device=f"cuda:{self.device}")
        st = (A.lodge_frame_stats * len(cl))()
        h = C.c_int64(0)
        A.call("lodge_render", self._h, int(sid), int(mode), camera_array(cl), len(cl),
               _ptr(out), _stream(stream), int(save), C.byref(h), st)
        imgs, off = [], 0
        flat = out.view(-1)
        for c in cl:
            n = c.width * c.height * 3
            imgs.append(flat[off:off + n].view(c.height, c.width, 3))
            off += n
        stats = [stats_dict(s) for s in st]
        res = (imgs[0] if single else imgs, stats[0] if single else stats)
        return res + (h.value,) if save else res

    def render_batch(self, frames, stream=None):
        """frames: list of (scene_id, mode, camera), composited by one launch.
        Returns (images, stats)."""
        n = len(frames)
        sids = (C.c_int32 * n)(*[int(f[0]) for f in frames])
        modes = (C.c_int32 * n)(*[int(f[1]) for f in frames])
        cams = camera_array([f[2] for f in frames])
        outs = [torch.empty(f[2].height, f[2].width, 3, dtype=torch.float32,
                            device=f"cuda:{self.device}") for f in frames]
        ptrs = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
        st = (A.lodge_frame_stats * n)()
        status = (C.c_int32 * n)()
        A.call("lodge_render_batch", self._h, n, sids, modes, cams, ptrs, _stream(stream), st, status)
        return outs, [stats_dict(s) for s in st]

    def render_host(self, sid: int, mode: int, cams, out: np.ndarray, stream=None):
        cl = list(cams)
        st = (A.lodge_frame_stats * len(cl))()
        A.call("lodge_render_host", self._h, int(sid), int(mode), camera_array(cl), len(cl),
               C.c_void_p(out.ctypes.data), _stream(stream), st)
        return [stats_dict(s) for s in st]

    def render_params(self, means, log_scales, quats, logits, sh, cam, sh_degree: int = 3,
                      filter_var: float = 0.0, stream=None, save: bool = True):
        for t in (means, log_scales, quats, logits, sh):
            assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
        out = torch.empty(cam.height, cam.width, 3, dtype=torch.float32, device=means.device)
        st = A.lodge_frame_stats()
        h = C.c_int64(0)
        A.call("lodge_render_params", self._h, int(means.shape[0]), _ptr(means), _ptr(log_scales),
               _ptr(quats), _ptr(logits), _ptr(sh), int(sh_degree), float(filter_var),
               C.byref(camera_struct(cam)), _ptr(out), _stream(stream), int(save), C.byref(h),
               C.byref(st))
        return out, stats_dict(st), (h.value if save else None)

    def render_params_lod(self, levels, cam, d_inner, filter_var, sh_degree: int = 3,
                          train_level: int = -1, score: Optional[torch.Tensor] = None,
                          stream=None, save: bool = False):
        """LOD render of levels given as device parameter tensors.

        levels: per level (finest first) a tuple (means (n,3), log_scales
        (n,3), quats (n,4), logits (n,), sh (n,48)) of contiguous float32
        cuda tensors; d_inner: this frame's thresholds d_1 .. d_{L-1};
        filter_var: per-level Eq. 3 variance.  score: optional importance
        accumulator over all levels' Gaussians (gid order).  save: keep the
        frame for render_backward (gradients of `train_level` only).
        Returns (image, stats, handle or None)."""
        L = len(levels)
        ptrs = [(C.c_void_p * L)() for _ in range(5)]
        ns = (C.c_int64 * L)()
        dev = None
        for l, lv in enumerate(levels):
            assert len(lv) == 5
            for k, t in enumerate(lv):
                assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
                ptrs[k][l] = t.data_ptr()
            ns[l] = int(lv[0].shape[0])
            dev = lv[0].device
        fv = (C.c_float * L)(*[float(v) for v in filter_var])
        d = np.ascontiguousarray(d_inner, np.float64).reshape(-1)
        assert d.size == L - 1
        out = torch.empty(cam.height, cam.width, 3, dtype=torch.float32, device=dev)
        st = A.lodge_frame_stats()
        h = C.c_int64(0)
        A.call("lodge_render_params_lod", self._h, L, ns, *ptrs, int(sh_degree), fv,
               C.c_void_p(d.ctypes.data) if d.size else None, C.byref(camera_struct(cam)), _ptr(out),
               _ptr(score), int(train_level), _stream(stream), int(save), C.byref(h), C.byref(st))
        return out, stats_dict(st), (h.value if save else None)

    def render_backward(self, handle: int, dL_drgb: torch.Tensor, g_means=None, g_log_scales=None,
                        g_quats=None, g_logits=None, g_sh=None, stream=None):
        A.call("lodge_render_backward", self._h, int(handle), _ptr(dL_drgb.contiguous()),
               _ptr(g_means), _ptr(g_log_scales), _ptr(g_quats), _ptr(g_logits), _ptr(g_sh),
               _stream(stream))

    def release(self, handle: int):
        A.call("lodge_release", self._h, int(handle))

    # -- inspection
    def debug_keys(self, handle: int, stream=None):
        n = C.c_int64(0)
        try:
            A.call("lodge_debug_keys", self._h, int(handle), None, None, 0, C.byref(n), _stream(stream))
        except LodgeError as e:
            if e.status != 7:
                raise
        dev = f"cuda:{self.device}"
        keys = torch.empty(max(n.value, 1), dtype=torch.int64, device=dev)
        gids = torch.empty(max(n.value, 1), dtype=torch.int32, device=dev)
        A.call("lodge_debug_keys", self._h, int(handle), _ptr(keys), _ptr(gids), n.value,
               C.byref(n), _stream(stream))
        return keys[:n.value], gids[:n.value]

    def debug_records(self, handle: int, stream=None):
        n = C.c_int64(0)
        try:
            A.call("lodge_debug_records", self._h, int(handle), None, None, None, None, None, None,
                   None, 0, C.byref(n), _stream(stream))
        except LodgeError as e:
            if e.status != 7:
                raise
        m = max(n.value, 1)
        dev = f"cuda:{self.device}"
        r = dict(gid=torch.empty(m, dtype=torch.int32, device=dev),
                 depth=torch.empty(m, dtype=torch.float32, device=dev),
                 rect=torch.empty(m, 4, dtype=torch.int32, device=dev),
                 mean2=torch.empty(m, 2, dtype=torch.float32, device=dev),
                 conic=torch.empty(m, 3, dtype=torch.float32, device=dev),
                 opacity=torch.empty(m, dtype=torch.float32, device=dev),
                 rgb=torch.empty(m, 3, dtype=torch.float32, device=dev))
        A.call("lodge_debug_records", self._h, int(handle), _ptr(r["gid"]), _ptr(r["depth"]),
               _ptr(r["rect"]), _ptr(r["mean2"]), _ptr(r["conic"]), _ptr(r["opacity"]),
               _ptr(r["rgb"]), n.value, C.byref(n), _stream(stream))
        return {k: v[:n.value] for k, v in r.items()}

    # -- serving and residency
    def serve(self, requests, slots: int = 4, realtime: bool = True, images: bool = False,
              wait_limit_s: float = 10.0, batch: int = 0):
        """requests: list of (scene_id, mode, camera, arrival_s).  batch > 0
        serves in steps composited by one launch each (at most batch frames).
        Returns (results list of dicts, images list or None).  Raises
        LodgeError only for invalid arguments; per-request failures are in
        each result."""
        n = len(requests)
        arr = (A.lodge_request * max(n, 1))()
        for i, (sid, mode, cam, t) in enumerate(requests):
            arr[i].scene = int(sid)
            arr[i].mode = int(mode)
            arr[i].cam = camera_struct(cam)
            arr[i].arrival_s = float(t)
        res = (A.lodge_request_result * max(n, 1))()
        opts = A.lodge_serve_opts()
        opts.slots = int(slots)
        opts.realtime = int(realtime)
        opts.wait_limit_s = float(wait_limit_s)
        opts.batch = int(batch)
        host = None
        if images:
            total = sum(c.width * c.height * 3 for _, _, c, _ in requests)
            host = np.zeros(max(total, 1), np.float32)
            opts.h_images = host.ctypes.data
        st = A.lib().lodge_serve(self._h, arr, n, C.byref(opts), res)
        if st not in (0, 1):
            A.check(st)
        out = []
        for i in range(n):
            r = res[i]
            out.append(dict(start_s=r.start_s, finish_s=r.finish_s, status=r.status, slot=r.slot,
                            latency_s=r.finish_s - requests[i][3], uploads=r.uploads,
                            step_frames=r.step_frames, **stats_dict(r.stats)))
        imgs = None
        if images:
            imgs, off = [], 0
            for _, _, c, _ in requests:
                k = c.width * c.height * 3
                imgs.append(host[off:off + k].reshape(c.height, c.width, 3))
                off += k
        return out, imgs

    def residency_stats(self) -> dict:
        r = A.lodge_residency()
        A.call("lodge_residency_stats", self._h, C.byref(r))
        return {f: getattr(r, f) for f, _ in r._fields_}

    def set_bin_size(self, log2_tiles: int):
        """Key lists per bin of 2**log2_tiles x 2**log2_tiles tiles (0..3),
        or -1 to choose per frame (the default); images do not depend on it
        (lodge_set_bin_size)."""
        A.call("lodge_set_bin_size", self._h, int(log2_tiles))

    def inject_upload_failures(self, n: int):
        A.call("lodge_inject_upload_failures", self._h, int(n))

    def profile_enable(self, enable: bool = True, count_pairs: bool = False):
        """Event timing per stage (counters reset); count_pairs: the counting
        mode (compositing counts its pixel-Gaussian pairs; times not plain)."""
        A.call("lodge_profile_enable", self._h, 2 if (enable and count_pairs) else int(enable))

    def profile_read(self) -> dict:
        p = A.lodge_profile()
        A.call("lodge_profile_read", self._h, C.byref(p))
        return dict(ms={n: p.ms[i] for i, n in enumerate(A.STAGE_NAMES)},
                    launches={n: p.launches[i] for i, n in enumerate(A.STAGE_NAMES)},
                    frames=p.frames, keys=p.keys, visible=p.visible, active=p.active,
                    packed_keys=p.packed_keys, bin_keys=p.bin_keys,
                    bin_sort_passes=p.bin_sort_passes, blend_pairs=p.blend_pairs,
                    blend_pairs_used=p.blend_pairs_used, redone=p.redone, host_ms=p.host_ms)

    def sort_pairs(self, keys: torch.Tensor, vals: torch.Tensor, key_bits: int = 32, stream=None):
        """Stable in-place sort of int32 (bit pattern = uint32) keys and values."""
        assert keys.dtype == torch.int32 and vals.dtype == torch.int32
        A.call("lodge_sort_pairs", self._h, _ptr(keys), _ptr(vals), int(keys.numel()), int(key_bits),
               _stream(stream))


def num_clusters(positions, d1: float) -> int:
    """Eq. 5: number of chunk clusters for camera positions (n x 3)."""
    p = np.ascontiguousarray(positions, np.float64).reshape(-1, 3)
    k = C.c_int32(0)
    A.call("lodge_num_clusters", C.c_void_p(p.ctypes.data), int(p.shape[0]), float(d1), C.byref(k))
    return k.value


def kmeans_centers(positions, init, max_iter: int = 100):
    """K-means chunk centres of camera positions from the given initial
    indices: (centres k x 3, assignment n, update steps)."""
    p = np.ascontiguousarray(positions, np.float64).reshape(-1, 3)
    ini = np.ascontiguousarray(init, np.int32)
    cen = np.zeros((ini.size, 3), np.float64)
    asg = np.zeros(p.shape[0], np.int32)
    it = C.c_int32(0)
    A.call("lodge_kmeans_centers", C.c_void_p(p.ctypes.data), int(p.shape[0]), int(ini.size),
           C.c_void_p(ini.ctypes.data), int(max_iter), C.c_void_p(cen.ctypes.data),
           C.c_void_p(asg.ctypes.data), C.byref(it))
    return cen, asg, it.value


class _RenderParams(torch.autograd.Function):
    """Differentiable render of raw Gaussian parameters through the library's
    forward (lodge_render_params) and hand-written adjoint
    (lodge_render_backward)."""

    @staticmethod
    def forward(fctx, means, log_scales, quats, logits, sh, lodge, cam, sh_degree, filter_var):
        img, stats, h = lodge.render_params(means, log_scales, quats, logits, sh, cam,
                                            sh_degree=sh_degree, filter_var=filter_var, save=True)
        fctx.lodge = lodge
        fctx.handle = h
        fctx.save_for_backward(means, log_scales, quats, logits, sh)
        return img

    @staticmethod
    def backward(fctx, g_img):
        means, log_scales, quats, logits, sh = fctx.saved_tensors
        gs = [torch.zeros_like(t) for t in (means, log_scales, quats, logits, sh)]
        try:
            fctx.lodge.render_backward(fctx.handle, g_img.contiguous(), *gs)
        finally:
            fctx.lodge.release(fctx.handle)
        return (*gs, None, None, None, None)


class _RenderLevelLod(torch.autograd.Function):
    """LOD render of several levels in which only one level's parameters are
    trained: forward lodge_render_params_lod, adjoint lodge_render_backward
    restricted to that level."""

    @staticmethod
    def forward(fctx, means, log_scales, quats, logits, sh, lodge, fixed, train_level, cam, d_inner,
                filter_var, sh_degree):
        trained = (means, log_scales, quats, logits, sh)
        levels = list(fixed[:train_level]) + [trained] + list(fixed[train_level:])
        img, stats, h = lodge.render_params_lod(levels, cam, d_inner, filter_var, sh_degree=sh_degree,
                                                train_level=train_level, save=True)
        fctx.lodge = lodge
        fctx.handle = h
        fctx.save_for_backward(*trained)
        return img

    @staticmethod
    def backward(fctx, g_img):
        trained = fctx.saved_tensors
        gs = [torch.zeros_like(t) for t in trained]
        try:
            fctx.lodge.render_backward(fctx.handle, g_img.contiguous(), *gs)
        finally:
            fctx.lodge.release(fctx.handle)
        return (*gs, None, None, None, None, None, None, None)


def render_level_lod(lodge: Lodge, trained, fixed, train_level: int, cam, d_inner, filter_var,
                     sh_degree: int = 3):
    """Image of an LOD frame over `fixed` levels plus the trained level
    (inserted at position train_level) that backpropagates to the trained
    level's five parameter tensors only."""
    return _RenderLevelLod.apply(*trained, lodge, list(fixed), int(train_level), cam, d_inner,
                                 list(filter_var), sh_degree)


def render_differentiable(lodge: Lodge, means, log_scales, quats, logits, sh, cam,
                          sh_degree: int = 3, filter_var: float = 0.0):
    """Image (H, W, 3) that backpropagates to the five parameter tensors."""
    return _RenderParams.apply(means, log_scales, quats, logits, sh, lodge, cam, sh_degree,
                               filter_var)
