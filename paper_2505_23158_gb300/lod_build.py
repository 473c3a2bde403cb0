"""Per-level LOD build (supplementary "LOD structure optimization steps";
Sec. 3 "Building LOD") on the library's render and adjoint.

Level l is made from the finest level G_0:
  1. copy G_0's parameters and give the copy the Eq. 3 smoothing filter of
     depth d_l (a per-level variance added to the covariance at render
     time; the parameters themselves are unchanged, so optimisation cannot
     shrink a Gaussian below the filter);
  2. three rounds, with importance thresholds 0.2 gamma, 0.6 gamma, gamma:
     a. score every Gaussian of the levels 0..l by its importance (the
        largest blending weight T alpha it receives, Sec. 3 "Importance
        pruning") over the views, rendering LOD frames with thresholds
        d_1 .. d_l, and prune the Gaussians of G_l scoring below the round's
        threshold (the finer levels are not pruned);
     b. run `steps` optimisation steps (the paper: 1000) of LOD rendering
        over the levels 0..l in which d_l is drawn from U(0.7 d_l, 1.3 d_l)
        per step, updating only G_l's parameters.
The loss is the one of the 3DGS training the paper keeps: (1 - lambda) L1 +
lambda (1 - SSIM), lambda = 0.2, SSIM over 11x11 Gaussian windows (sigma 1.5)
per channel (`dssim_l1`; lambda = 0 gives plain L1).  Adam drives the
updates; the render, the importance walk and the gradients of the image are
the library's kernels (lodge_render_params_lod, lodge_render_backward); the
loss and its gradient with respect to the image are torch operations.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence

import numpy as np
import torch

from .api import Lodge, render_level_lod

ROUND_FRACTIONS = (0.2, 0.6, 1.0)
SSIM_WEIGHT = 0.2      # lambda of the 3DGS loss


def _gauss_window(size: int = 11, sigma: float = 1.5, device=None) -> torch.Tensor:
    x = torch.arange(size, dtype=torch.float32, device=device) - (size - 1) / 2
    g = torch.exp(-x * x / (2 * sigma * sigma))
    g = g / g.sum()
    return (g[:, None] * g[None, :])[None, None]        # (1, 1, size, size)


def ssim(img: torch.Tensor, ref: torch.Tensor, size: int = 11, sigma: float = 1.5) -> torch.Tensor:
    """Mean SSIM of two (H, W, 3) images in [0, 1]: per channel, local means,
    variances and covariance under a Gaussian window (zero padding, "same"
    size), C1 = 0.01^2, C2 = 0.03^2, averaged over pixels and channels."""
    x = img.permute(2, 0, 1)[:, None]                       # (3, 1, H, W)
    y = ref.permute(2, 0, 1)[:, None]
    w = _gauss_window(size, sigma, img.device)
    pad = size // 2
    f = lambda t: torch.nn.functional.conv2d(t, w, padding=pad)
    mx, my = f(x), f(y)
    sxx = f(x * x) - mx * mx
    syy = f(y * y) - my * my
    sxy = f(x * y) - mx * my
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    s = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
    return s.mean()


def dssim_l1(img: torch.Tensor, ref: torch.Tensor, lam: float = SSIM_WEIGHT) -> torch.Tensor:
    """(1 - lam) L1 + lam (1 - SSIM) of an image against its target."""
    l1 = (img - ref).abs().mean()
    if lam == 0.0:
        return l1
    return (1.0 - lam) * l1 + lam * (1.0 - ssim(img, ref))


def level_params(level, device) -> tuple:
    """A synth.Level's raw parameters as contiguous float32 cuda tensors
    (means, log_scales, quats, logits, sh (n, 48))."""
    n = level.n
    arrs = (level.means, level.log_scales, level.quats, level.opacity_logits,
            np.asarray(level.sh, np.float32).reshape(n, 48))
    return tuple(torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device) for a in arrs)


def filter_variance(scale: float, depth: float, focal: float) -> float:
    """Eq. 3 smoothing filter of depth d for a camera of focal length f
    (pixels), read as a variance: (s d / f)^2."""
    return float((scale * depth / focal) ** 2)


def importance_scores(ctx: Lodge, levels: Sequence[tuple], views, d_inner, filter_var,
                      sh_degree: int = 3) -> torch.Tensor:
    """Largest blending weight of every Gaussian of `levels` (gid order,
    finest first) over LOD renders of the views at thresholds d_inner."""
    n = sum(int(l[0].shape[0]) for l in levels)
    score = torch.zeros(max(n, 1), dtype=torch.float32, device=levels[0][0].device)
    for cam in views:
        ctx.render_params_lod(list(levels), cam, d_inner, filter_var, sh_degree=sh_degree, score=score)
    return score[:n]


EVAL_FACTORS = (0.7, 0.85, 1.0, 1.15, 1.3)


def eval_loss(ctx: Lodge, fixed, trained, l: int, views, targets, d, filter_var, sh_degree: int = 3,
              lam: float = SSIM_WEIGHT) -> float:
    """The objective the steps sample, evaluated deterministically: the mean
    loss (dssim_l1) over the views and over d_l at 0.7, 0.85, 1.0, 1.15 and
    1.3 of its nominal value (the other thresholds fixed)."""
    levels = list(fixed[:l]) + [tuple(trained)] + list(fixed[l:])
    d = np.asarray(d, np.float64)
    tot, cnt = 0.0, 0
    for f in EVAL_FACTORS:
        dd = d.copy()
        dd[-1] = f * d[-1]
        for cam, tgt in zip(views, targets):
            img, _, _ = ctx.render_params_lod(levels, cam, dd, filter_var, sh_degree=sh_degree)
            tot += float(dssim_l1(img, tgt, lam))
            cnt += 1
    return tot / max(cnt, 1)


def build_level(ctx: Lodge, fixed: Sequence[tuple], base: tuple, d: Sequence[float], views,
                targets: Sequence[torch.Tensor], gamma: float, filter_var_l: float,
                filter_var_fixed: Sequence[float], steps: int = 1000, lr: Optional[dict] = None,
                seed: int = 0, sh_degree: int = 3, keep_params: bool = False, lam: float = SSIM_WEIGHT,
                on_round: Optional[Callable[[int, dict], None]] = None):
    """Build level l = len(fixed) from `base` (G_0's parameters).

    fixed: parameters of levels 0 .. l-1 (not updated); d: thresholds
    d_1 .. d_l; views / targets: cameras and their target images (H, W, 3);
    gamma: importance threshold of the last round; filter_var_l /
    filter_var_fixed: Eq. 3 variances of the new and the fixed levels;
    lam: the SSIM weight of the loss (0: plain L1).
    Returns (parameters of G_l, history) where history holds per round the
    threshold, the scores of G_l before pruning, the kept count, the loss of
    every step, and the objective (eval_loss) after pruning and after the
    round's steps (and, with keep_params, host
    copies of the parameters that were scored and of those after the
    round's steps)."""
    l = len(fixed)
    assert len(d) == l and l >= 1
    # fine-tuning rates (the tail of a 3DGS schedule: small position steps)
    lr = lr or {"means": 1e-5, "log_scales": 2e-3, "quats": 5e-4, "logits": 1e-2, "sh": 1e-3}
    rng = np.random.default_rng(seed)
    fvs = list(filter_var_fixed) + [filter_var_l]
    d = np.asarray(d, np.float64)
    cur = [t.clone() for t in base]
    off = sum(int(f[0].shape[0]) for f in fixed)
    history: List[dict] = []
    for r, frac in enumerate(ROUND_FRACTIONS):
        thr = frac * gamma
        score = importance_scores(ctx, list(fixed) + [tuple(cur)], views, d, fvs, sh_degree)
        s_l = score[off:off + int(cur[0].shape[0])]
        scored = [t.cpu().numpy() for t in cur] if keep_params else None
        keep = s_l >= thr
        cur = [t[keep].contiguous() for t in cur]
        loss_pruned = eval_loss(ctx, fixed, cur, l, views, targets, d, fvs, sh_degree, lam)
        params = [t.detach().clone().requires_grad_(True) for t in cur]
        names = ("means", "log_scales", "quats", "logits", "sh")
        opt = torch.optim.Adam([{"params": [p], "lr": lr[k]} for p, k in zip(params, names)], eps=1e-15)
        # rates decay exponentially to a tenth over the round's steps
        sched = torch.optim.lr_scheduler.LambdaLR(opt, lambda t: 0.1 ** (t / max(steps, 1)))
        losses = []
        for step in range(steps):
            i = step % len(views)
            dd = d.copy()
            dd[-1] = rng.uniform(0.7, 1.3) * d[-1]
            img = render_level_lod(ctx, params, fixed, l, views[i], dd, fvs, sh_degree)
            loss = dssim_l1(img, targets[i], lam)
            opt.zero_grad(set_to_none=True)
            loss.backward()
            opt.step()
            sched.step()
            losses.append(float(loss.detach()))
        cur = [p.detach().contiguous() for p in params]
        loss_tuned = eval_loss(ctx, fixed, cur, l, views, targets, d, fvs, sh_degree, lam)
        rec = {"round": r, "threshold": thr, "scores": s_l.detach().cpu().numpy(),
               "kept": int(keep.sum()), "losses": np.asarray(losses),
               "loss_pruned": loss_pruned, "loss_tuned": loss_tuned}
        if keep_params:
            rec["scored_params"] = scored
            rec["params"] = [t.cpu().numpy() for t in cur]
        history.append(rec)
        if on_round:
            on_round(r, rec)
    return tuple(cur), history
