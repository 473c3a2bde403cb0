"""CPU oracle for the LODGE per-frame render path (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  It never imports the CUDA
package and the CUDA package never imports it.  The numerical work lives in
``oracle.c`` (FP64, with the FP32 key spec for integer decisions); this file
compiles it with gcc and marshals numpy arrays into it.

Public functions mirror the paper's steps:
  activate            3DGS activations (exp, sigmoid, unit quaternion)
  chunk_radius        distance to the nearest other chunk centre (Sec. 3)
  chunk_pick          two nearest chunk centres and Eq. 4 weights
  lod_select          Eq. 2 active set at a centre
  chunk_select        Eq. 2 at a chunk centre with offset thresholds (Sec. 3)
  chunk_union         union of two chunk sets with Eq. 4 multipliers
  active_set          the active list for a render mode and camera
  project / keys      per-Gaussian projection records, sorted tile keys
  n_keys              number of tile keys of an active list
  importance          largest blending weight per Gaussian in a view (Sec. 3)
  render              Eq. 1 compositing (binned or brute force), with the range
                      of results over FP32-reachable knife-edge decisions
  compare_pixels      the pixel bar against render's result and ranges
  select_thresholds   greedy depth-threshold search (Sec. 3)
  num_clusters        number of chunk clusters (supplementary Eq. 5)
  kmeans_centers      K-means chunk centres from camera positions
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_FULL, MODE_LOD, MODE_CHUNK, MODE_CHUNK_BLEND = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, FP64, no FMA
    contraction, OpenMP over tiles)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float),
                ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32), ("znear", C.c_float),
                ("pad_", C.c_float), ("center", C.c_double * 3)]


class _Scene(C.Structure):
    _fields_ = [("n_total", C.c_int64), ("num_levels", C.c_int32), ("sh_degree", C.c_int32),
                ("level_off", C.c_void_p), ("filter_var", C.c_void_p), ("means", C.c_void_p),
                ("scales", C.c_void_p), ("quats", C.c_void_p), ("opac", C.c_void_p),
                ("sh", C.c_void_p), ("filter2d", C.c_int32)]


class _Stats(C.Structure):
    _fields_ = [("n_visible", C.c_int64), ("n_keys", C.c_int64), ("n_pairs_eval", C.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.c_void_p
            lib.orc_activate.argtypes = [C.c_int64, P, P, P, P, P, P]
            lib.orc_chunk_radius.argtypes = [C.c_int32, P, P]
            lib.orc_chunk_pick.argtypes = [C.c_int32, P, P, P, P, P, P]
            lib.orc_chunk_tsum_unclamped.argtypes = [P, P, P]
            lib.orc_chunk_tsum_unclamped.restype = C.c_double
            lib.orc_lod_select.argtypes = [P, P, P, P, P]
            lib.orc_lod_select.restype = C.c_int64
            lib.orc_chunk_select.argtypes = [P, C.c_int32, P, P, C.c_int32, P, P]
            lib.orc_chunk_select.restype = C.c_int64
            lib.orc_chunk_union.argtypes = [C.c_int64, P, C.c_int64, P, C.c_double,
                                            C.c_double, P, P]
            lib.orc_chunk_union.restype = C.c_int64
            lib.orc_render.argtypes = [P, P, C.c_int64, P, P, C.c_int32, P, C.c_int32,
                                       C.c_double, C.c_double, P, P, P, P, P, P, P]
            lib.orc_project.argtypes = [P, P, C.c_int64, P, P, P, P, P, P, P, P, P, P, P]
            lib.orc_importance.argtypes = [P, P, C.c_int64, P, P, C.c_double, C.c_double, P, P]
            lib.orc_keys.argtypes = [P, P, C.c_int64, P, P, P, P, C.c_int64]
            lib.orc_keys.restype = C.c_int64
            lib.orc_sh_basis.argtypes = [C.c_double, C.c_double, C.c_double, P]
            lib.orc_depth32.argtypes = [P, P, C.c_int64, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
def activate(log_scales, quats, logits):
    """scale = exp(log_scale), unit quaternion, opacity = sigmoid(logit),
    computed in FP64 and rounded once to FP32."""
    lib = _load()
    ls = _c(log_scales, np.float32); q = _c(quats, np.float32); lg = _c(logits, np.float32)
    n = ls.shape[0]
    s = np.empty((n, 3), np.float32); qn = np.empty((n, 4), np.float32); o = np.empty(n, np.float32)
    lib.orc_activate(n, _p(ls), _p(q), _p(lg), _p(s), _p(qn), _p(o))
    return s, qn, o


class OracleScene:
    """Activated, level-concatenated copy of a synthetic scene.  gid = global
    index into the concatenation (level-major), so gid order is level order,
    then index order within a level."""

    def __init__(self, scene):
        lv = scene.levels
        self.num_levels = len(lv)
        self.level_off = np.zeros(len(lv) + 1, np.int64)
        for i, l in enumerate(lv):
            self.level_off[i + 1] = self.level_off[i] + l.n
        self.n_total = int(self.level_off[-1])
        self.means = _c(np.concatenate([l.means for l in lv]), np.float32)
        s, q, o = activate(np.concatenate([l.log_scales for l in lv]),
                           np.concatenate([l.quats for l in lv]),
                           np.concatenate([l.opacity_logits for l in lv]))
        self.scales, self.quats, self.opac = s, q, o
        self.sh = _c(np.concatenate([l.sh for l in lv]), np.float32)
        self.filter_var = np.array([l.filter_var for l in lv], np.float32)
        self.sh_degree = int(scene.sh_degree)
        self.d_inner = np.asarray(scene.d_thresholds, np.float64)
        self.centers = _c(scene.chunk_centers, np.float64)
        self._s = _Scene(self.n_total, self.num_levels, self.sh_degree,
                         self.level_off.ctypes.data, self.filter_var.ctypes.data,
                         self.means.ctypes.data, self.scales.ctypes.data,
                         self.quats.ctypes.data, self.opac.ctypes.data, self.sh.ctypes.data,
                         int(bool(getattr(scene, "filter2d", False))))
        self._chunk_cache = {}

    @property
    def ptr(self):
        return C.byref(self._s)


def _cam(cam) -> _Camera:
    c = _Camera()
    c.R[:] = [float(x) for x in np.asarray(cam.R, np.float32).ravel()]
    c.t[:] = [float(x) for x in np.asarray(cam.t, np.float32).ravel()]
    c.fx, c.fy, c.cx, c.cy = (float(np.float32(cam.fx)), float(np.float32(cam.fy)),
                              float(np.float32(cam.cx)), float(np.float32(cam.cy)))
    c.width, c.height = int(cam.width), int(cam.height)
    c.znear = float(np.float32(cam.znear))
    c.center[:] = [float(x) for x in np.asarray(cam.center, np.float64)]
    return c


# --------------------------------------------------------------------------
def chunk_radius(centers):
    lib = _load()
    c = _c(centers, np.float64)
    r = np.empty(c.shape[0], np.float64)
    lib.orc_chunk_radius(c.shape[0], _p(c), _p(r))
    return r


def chunk_pick(centers, c):
    """(A, B, t_A, t_B) for camera position c (Eq. 4)."""
    lib = _load()
    cc = _c(centers, np.float64)
    pos = _c(c, np.float64)
    A = C.c_int32(); B = C.c_int32(); tA = C.c_double(); tB = C.c_double()
    lib.orc_chunk_pick(cc.shape[0], _p(cc), _p(pos), C.byref(A), C.byref(B),
                       C.byref(tA), C.byref(tB))
    return A.value, B.value, tA.value, tB.value


def chunk_tsum_unclamped(mA, mB, c):
    lib = _load()
    a, b, p = _c(mA, np.float64), _c(mB, np.float64), _c(c, np.float64)
    return lib.orc_chunk_tsum_unclamped(_p(a), _p(b), _p(p))


def lod_select(osc: OracleScene, c, d_inner=None):
    """Eq. 2 at centre c; returns (gids int64 ascending, n_disagree_fp64)."""
    lib = _load()
    d = osc.d_inner if d_inner is None else _c(d_inner, np.float64)
    d = _c(d, np.float64)
    pos = _c(c, np.float64)
    mask = np.zeros(osc.n_total, np.uint8)
    dis = C.c_int64()
    lib.orc_lod_select(osc.ptr, _p(pos), _p(d) if d.size else None, _p(mask), C.byref(dis))
    return np.flatnonzero(mask).astype(np.int64), dis.value


def chunk_select(osc: OracleScene, k: int):
    """Active set of chunk k: Eq. 2 at m_k with thresholds d_l + r_k."""
    if k in osc._chunk_cache:
        return osc._chunk_cache[k]
    lib = _load()
    mask = np.zeros(osc.n_total, np.uint8)
    dis = C.c_int64()
    d = _c(osc.d_inner, np.float64)
    lib.orc_chunk_select(osc.ptr, osc.centers.shape[0], _p(osc.centers),
                         _p(d) if d.size else None, int(k), _p(mask), C.byref(dis))
    res = np.flatnonzero(mask).astype(np.int64)
    osc._chunk_cache[k] = res
    return res


def chunk_union(a, b, tA, tB):
    lib = _load()
    a = _c(a, np.int64); b = _c(b, np.int64)
    out = np.empty(a.size + b.size, np.int64); mult = np.empty(a.size + b.size, np.float32)
    n = lib.orc_chunk_union(a.size, _p(a), b.size, _p(b), float(tA), float(tB), _p(out), _p(mult))
    return out[:n].copy(), mult[:n].copy()


def active_set(osc: OracleScene, mode: int, cam):
    """(gids, mults, info) for one camera.
    FULL: every level-0 Gaussian.  LOD: Eq. 2 at the camera centre.
    CHUNK: the nearest chunk's set.  CHUNK_BLEND: union of the two nearest
    chunks' sets with Eq. 4 multipliers."""
    info = {}
    if mode == MODE_FULL:
        g = np.arange(osc.level_off[1], dtype=np.int64)
        return g, None, info
    if mode == MODE_LOD:
        g, dis = lod_select(osc, cam.center)
        info["n_disagree"] = dis
        return g, None, info
    A, B, tA, tB = chunk_pick(osc.centers, cam.center)
    info.update(A=A, B=B, tA=tA, tB=tB)
    if mode == MODE_CHUNK or B < 0:
        return chunk_select(osc, A), None, info
    g, m = chunk_union(chunk_select(osc, A), chunk_select(osc, B), tA, tB)
    return g, m, info


# FP32 error model of the renderer under test (orc_fp32_err in oracle.c): the
# pixel offset d = p - mu' is off by at most ERR_DD pixels (about four ulp of
# a 3840-pixel coordinate, the largest image of the workloads), and alpha by a
# relative 1e-5 from everything else.  Only used to find knife-edge decisions.
ERR_DD = 1e-3
ERR_KE0 = 1e-5


def render(osc: OracleScene, cam, gids, mults=None, brute=False, tiles=None,
           err_dd=ERR_DD, err_ke0=ERR_KE0, bounds=True):
    """Composite the active list; returns dict(rgb (H,W,3) f64, T, ncontrib,
    knife, knife_code, lo, hi, n_visible, n_keys, n_pairs_eval).

    ``rgb`` takes every Eq. 1 decision (the 1/255 skip, the 1e-4 stop) as
    FP64 does.  Where FP32 rounding may take one the other way (knife edge,
    ``knife_code`` 1), every such choice gives a correct render, and ``lo`` /
    ``hi`` bound the results over all of them per channel; ``knife_code`` 2
    marks pixels with more decision paths than the oracle enumerates."""
    lib = _load()
    H, W = int(cam.height), int(cam.width)
    g = _c(gids, np.int64)
    m = None if mults is None else _c(mults, np.float32)
    t = None if tiles is None else _c(tiles, np.int32)
    rgb = np.zeros((H, W, 3), np.float64); T = np.ones((H, W), np.float64)
    nc = np.zeros((H, W), np.int32); kn = np.zeros((H, W), np.uint8)
    lo = np.zeros((H, W, 3), np.float64) if bounds else None
    hi = np.zeros((H, W, 3), np.float64) if bounds else None
    st = _Stats()
    cc = _cam(cam)
    lib.orc_render(osc.ptr, C.byref(cc), g.size, _p(g), None if m is None else _p(m),
                   1 if brute else 0, None if t is None else _p(t),
                   0 if t is None else t.size, float(err_dd), float(err_ke0),
                   _p(rgb), _p(T), _p(nc), _p(kn), None if lo is None else _p(lo),
                   None if hi is None else _p(hi), C.byref(st))
    return dict(rgb=rgb, T=T, ncontrib=nc, knife=kn.astype(bool), knife_code=kn, lo=lo, hi=hi,
                n_visible=st.n_visible, n_keys=st.n_keys, n_pairs_eval=st.n_pairs_eval)


def compare_pixels(img, ref, mask=None, max_abs=2e-4, mean_abs=1e-5, unresolved_frac=1e-5):
    """Check an image against ``render``'s result on clamp(rgb, 0, 1).

    Pixels without a knife-edge decision must be within ``max_abs`` of the
    oracle per channel; knife-edge pixels within ``max_abs`` of the range
    [lo, hi] of the results their FP32-reachable decisions give; the mean
    of those distances over all pixels must be at most ``mean_abs``.  Pixels
    whose decision paths exceed the enumeration (``knife_code`` 2) are left
    out of the max and may be at most ``unresolved_frac`` of the pixels.
    ``mask`` (H, W) restricts the check.  Returns the counts and errors;
    raises AssertionError when a bar is missed."""
    g = np.clip(np.asarray(img, np.float64), 0, 1)
    r = np.clip(ref["rgb"], 0, 1)
    code = ref["knife_code"]
    if ref["lo"] is None:
        raise ValueError("compare_pixels needs render(..., bounds=True)")
    lo = np.clip(ref["lo"], 0, 1); hi = np.clip(ref["hi"], 0, 1)
    if mask is not None:
        g, r, code, lo, hi = g[mask], r[mask], code[mask], lo[mask], hi[mask]
    g = g.reshape(-1, 3); r = r.reshape(-1, 3); lo = lo.reshape(-1, 3); hi = hi.reshape(-1, 3)
    code = code.reshape(-1)
    plain = np.abs(g - r)
    env = np.maximum(np.maximum(lo - g, g - hi), 0.0)
    dist = np.where((code == 0)[:, None], plain, np.where((code == 1)[:, None], env, plain))
    checked = code != 2
    worst = float(dist[checked].max()) if checked.any() else 0.0
    mean = float(dist.mean()) if dist.size else 0.0
    n_pix = int(code.size)
    out = dict(pixels=n_pix, knife=int((code > 0).sum()), unresolved=int((code == 2).sum()),
               took_other=int(((code == 1) & (plain.max(axis=1) > max_abs)).sum()),
               max_abs=worst, mean_abs=mean, mean_abs_plain=float(plain.mean()) if plain.size else 0.0)
    bad = []
    if worst > max_abs:
        i = int(np.argmax(np.where(checked[:, None], dist, 0).max(axis=1)))
        bad.append(f"max-abs {worst:.3g} at pixel {i} (knife code {int(code[i])})")
    if mean > mean_abs:
        bad.append(f"mean-abs {mean:.3g}")
    if out["unresolved"] > math.floor(unresolved_frac * n_pix):
        bad.append(f"{out['unresolved']} unresolved knife-edge pixels")
    if bad:
        raise AssertionError("; ".join(bad) + f" ({out})")
    return out


def project(osc: OracleScene, cam, gids, mults=None):
    lib = _load()
    g = _c(gids, np.int64)
    n = g.size
    m = None if mults is None else _c(mults, np.float32)
    out = dict(visible=np.zeros(n, np.uint8), z=np.zeros(n, np.float32),
               rect=np.zeros((n, 4), np.int32), o32=np.zeros(n, np.float32),
               mean2=np.zeros((n, 2)), conic=np.zeros((n, 3)), cov=np.zeros((n, 3)),
               opacity=np.zeros(n), rgb=np.zeros((n, 3)))
    cc = _cam(cam)
    lib.orc_project(osc.ptr, C.byref(cc), n, _p(g), None if m is None else _p(m),
                    _p(out["visible"]), _p(out["z"]), _p(out["rect"]), _p(out["o32"]),
                    _p(out["mean2"]), _p(out["conic"]), _p(out["cov"]), _p(out["opacity"]),
                    _p(out["rgb"]))
    out["visible"] = out["visible"].astype(bool)
    return out


def keys(osc: OracleScene, cam, gids, mults=None):
    """Sorted (tile << 32 | depth bits) keys and the gid of each key."""
    lib = _load()
    g = _c(gids, np.int64)
    m = None if mults is None else _c(mults, np.float32)
    cc = _cam(cam)
    n = lib.orc_keys(osc.ptr, C.byref(cc), g.size, _p(g), None if m is None else _p(m),
                     None, None, 0)
    k = np.empty(n, np.uint64); gg = np.empty(n, np.int64)
    lib.orc_keys(osc.ptr, C.byref(cc), g.size, _p(g), None if m is None else _p(m),
                 _p(k), _p(gg), n)
    return k, gg


def importance(osc: OracleScene, cam, gids, mults=None, ke_alpha=1e-4, ke_t=1e-4):
    """Importance score of each active entry for one view (Sec. 3, after
    RadSplat): the largest blending weight T * alpha it receives at any
    pixel where it is composited (0 if never).  Returns (score, clean):
    ``clean`` takes the maximum only over pixels without a knife-edge
    decision (alpha near 1/255 or T near 1e-4), where FP32 and FP64 can
    composite different entries."""
    lib = _load()
    g = _c(gids, np.int64)
    m = None if mults is None else _c(mults, np.float32)
    sa = np.zeros(g.size, np.float64)
    sc = np.zeros(g.size, np.float64)
    cc = _cam(cam)
    lib.orc_importance(osc.ptr, C.byref(cc), g.size, _p(g), None if m is None else _p(m),
                       float(ke_alpha), float(ke_t), _p(sa), _p(sc))
    return sa, sc


def n_keys(osc: OracleScene, cam, gids, mults=None) -> int:
    """Number of (tile, Gaussian) keys of an active list: the sum over its
    visible Gaussians of the tiles their rect covers."""
    lib = _load()
    g = _c(gids, np.int64)
    m = None if mults is None else _c(mults, np.float32)
    cc = _cam(cam)
    return int(lib.orc_keys(osc.ptr, C.byref(cc), g.size, _p(g), None if m is None else _p(m),
                            None, None, 0))


def select_thresholds(osc: OracleScene, views, candidates):
    """Greedy depth-threshold search (Sec. 3, "Selecting depth thresholds").

    The cost of a threshold set is the number of Gaussians summed over the
    16x16 tiles of the views, i.e. the tile keys of LOD rendering (Eq. 2 at
    each camera centre), summed over the views.  Reading of the greedy
    strategy: thresholds are added one at a time, starting with d_1; when
    d_l is searched, d_1 .. d_{l-1} are fixed and levels above l are not used
    (d_{l+1} = ... = inf), and d_l is the candidate larger than d_{l-1} with
    the least cost, the smaller one on ties.  If no candidate is left, d_l
    and the later thresholds are inf.

    Returns (d, table): d the L-1 thresholds, table[l-1, k] the cost of
    candidate k at step l (-1 where it was not eligible)."""
    cand = [float(x) for x in candidates]
    L = osc.num_levels
    d = []
    table = np.full((max(L - 1, 0), len(cand)), -1, np.int64)
    for l in range(1, L):
        prev = d[-1] if d else 0.0
        if math.isinf(prev):
            d.append(math.inf)
            continue
        for k, x in enumerate(cand):
            if not x > prev:
                continue
            thresholds = d + [x] + [math.inf] * (L - 1 - l)
            total = 0
            for cam in views:
                g, _ = lod_select(osc, cam.center, thresholds)
                total += n_keys(osc, cam, g)
            table[l - 1, k] = total
        row = table[l - 1]
        ok = np.flatnonzero(row >= 0)
        if ok.size == 0:
            d.append(math.inf)
            continue
        best = ok[np.argmin(row[ok])]     # argmin returns the first minimum
        d.append(cand[best])
    return d, table


def num_clusters(positions, d1: float) -> int:
    """Eq. 5 (supplementary "Selecting chunk centers"):
    N = (4 / d_1) max_i |c_i - c_mean|, read as the ceiling, clamped to
    [1, number of cameras].  The mean sums the positions in index order."""
    p = np.asarray(positions, np.float64).reshape(-1, 3)
    mean = [0.0, 0.0, 0.0]
    for row in p:
        for c in range(3):
            mean[c] += float(row[c])
    mean = [v / p.shape[0] for v in mean]
    rmax = 0.0
    for row in p:
        dx, dy, dz = row[0] - mean[0], row[1] - mean[1], row[2] - mean[2]
        rmax = max(rmax, math.sqrt((dx * dx + dy * dy) + dz * dz))
    k = math.ceil(4.0 / d1 * rmax)
    return int(min(max(k, 1), p.shape[0]))


def _nearest(p, m):
    best, bd = 0, None
    for j in range(m.shape[0]):
        dx, dy, dz = p[0] - m[j, 0], p[1] - m[j, 1], p[2] - m[j, 2]
        d = (dx * dx + dy * dy) + dz * dz
        if bd is None or d < bd:
            best, bd = j, d
    return best


def kmeans_centers(positions, init, max_iter: int = 100):
    """K-means (Lloyd) on camera positions (supplementary "Selecting chunk
    centers"; the paper names the method, these are its textbook steps):
    centres start at the positions of ``init``; each step assigns every
    position to its nearest centre (ties to the lower index) and stops if no
    assignment changed, else moves each centre to the mean of its positions
    (a centre without positions stays).  Returns (centres, assignment to the
    returned centres, number of update steps)."""
    p = np.asarray(positions, np.float64).reshape(-1, 3)
    m = p[np.asarray(init, np.int64)].copy()
    a = [-1] * p.shape[0]
    it = 0
    while it < max_iter:
        new = [_nearest(p[i], m) for i in range(p.shape[0])]
        if new == a:
            break
        a = new
        for j in range(m.shape[0]):
            members = [i for i in range(p.shape[0]) if a[i] == j]
            if not members:
                continue
            acc = [0.0, 0.0, 0.0]
            for i in members:           # index order
                for c in range(3):
                    acc[c] += float(p[i, c])
            m[j] = [v / len(members) for v in acc]
        it += 1
    assign = np.array([_nearest(p[i], m) for i in range(p.shape[0])], np.int32)
    return m, assign, it


def depth32(means, cam):
    """FP32 key depth (camera z by the key spec) of each mean."""
    lib = _load()
    m = _c(means, np.float32)
    z = np.empty(m.shape[0], np.float32)
    cc = _cam(cam)
    lib.orc_depth32(_p(m), C.byref(cc), m.shape[0], _p(z))
    return z


def sh_basis(d):
    lib = _load()
    Y = np.empty(16, np.float64)
    lib.orc_sh_basis(float(d[0]), float(d[1]), float(d[2]), _p(Y))
    return Y
