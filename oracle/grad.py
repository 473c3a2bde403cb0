"""FP64 gradient oracle of the render path (test infrastructure).

A plain PyTorch CPU forward of the same definition as oracle.c, written for
differentiation: every Gaussian in front of the near plane is evaluated at
every pixel (brute force), in (FP32 key depth, index) order, and
torch.autograd differentiates it in FP64.  Used to check the CUDA adjoint
(fine-tuning of a level, supplementary "LOD structure optimization steps":
the levels are optimised with gradients through the renderer).

Steps, in the paper's and 3DGS's order (see oracle.c for each reading):
  activation: s = exp(log s), o = sigmoid(logit), unit quaternion;
  Eq. 3 filter: Sigma = R(q) diag(s^2 + v) R(q)^T, o *= prod s / sqrt(s^2 + v);
  EWA: p = R mu + t, J (at x/z, y/z clamped to 1.3 tan(fov/2)), Sigma' = J W Sigma W^T J^T + 0.3 I, mean' in pixels;
  colour: real SH up to degree 3 at (mu - c)/|mu - c|, + 0.5, clamped at 0;
  Eq. 1: alpha = min(0.99, o' exp(-1/2 d^T Sigma'^-1 d)), skip alpha < 1/255,
  stop before T would drop below 1e-4, C = sum T alpha rgb.
The discrete decisions (skip, stop) are taken on the FP64 values and held
fixed under differentiation, as the renderer's own adjoint does.

Pinned by tests/test_oracle_grad.py: its image equals oracle.c's render, and
its gradients equal central finite differences of itself.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import depth32

PI = math.pi


def sh_basis_t(d: torch.Tensor) -> torch.Tensor:
    """Real orthonormal SH basis up to l = 3 for unit directions d (N, 3)."""
    x, y, z = d[:, 0], d[:, 1], d[:, 2]
    c0 = 0.5 * math.sqrt(1.0 / PI)
    c1 = math.sqrt(3.0 / (4.0 * PI))
    Y = [torch.full_like(x, c0), c1 * y, c1 * z, c1 * x,
         0.5 * math.sqrt(15.0 / PI) * x * y,
         0.5 * math.sqrt(15.0 / PI) * y * z,
         0.25 * math.sqrt(5.0 / PI) * (3 * z * z - 1),
         0.5 * math.sqrt(15.0 / PI) * x * z,
         0.25 * math.sqrt(15.0 / PI) * (x * x - y * y),
         0.25 * math.sqrt(35.0 / (2 * PI)) * y * (3 * x * x - y * y),
         0.5 * math.sqrt(105.0 / PI) * x * y * z,
         0.25 * math.sqrt(21.0 / (2 * PI)) * y * (5 * z * z - 1),
         0.25 * math.sqrt(7.0 / PI) * z * (5 * z * z - 3),
         0.25 * math.sqrt(21.0 / (2 * PI)) * x * (5 * z * z - 1),
         0.25 * math.sqrt(105.0 / PI) * z * (x * x - y * y),
         0.25 * math.sqrt(35.0 / (2 * PI)) * x * (x * x - 3 * y * y)]
    return torch.stack(Y, dim=1)


def quat_to_rot(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrices (N, 3, 3) of unit quaternions (w, x, y, z)."""
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], 1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], 1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1),
    ], 1)


def render_t(means, log_scales, quats, logits, sh, cam, sh_degree=3, filter_var=0.0,
             mults=None, order=None, pix_chunk=1024, return_aux=False):
    """Image (H, W, 3) from raw parameters (torch tensors, FP64 -- or FP32
    to measure how much rounding at that precision moves a result -- possibly
    requiring grad).  `order`: Gaussian indices in compositing order
    (default: by FP32 key depth then index, near-culled ones dropped)."""
    H, W = int(cam.height), int(cam.width)
    ft = means.dtype
    nf = np.float64 if ft == torch.float64 else np.float32
    if order is None:
        z32 = depth32(means.detach().to(torch.float32).numpy(), cam)
        idx = np.arange(z32.size)
        keep = z32 > np.float32(cam.znear)
        o = np.lexsort((idx[keep], z32[keep]))
        order = idx[keep][o]
    order_t = torch.as_tensor(order, dtype=torch.long)
    mu = means[order_t]
    s = torch.exp(log_scales[order_t])
    qr = quats[order_t]
    q = qr / torch.linalg.norm(qr, dim=1, keepdim=True)
    op = torch.sigmoid(logits[order_t])
    if mults is not None:
        op = op * torch.as_tensor(np.asarray(mults, np.float64)[order], dtype=ft)
    v = float(filter_var)
    s2 = s * s + v
    if v > 0:
        op = op * torch.prod(s / torch.sqrt(s2), dim=1)
    Rq = quat_to_rot(q)
    Sig = Rq @ torch.diag_embed(s2) @ Rq.transpose(1, 2)
    R = torch.as_tensor(np.asarray(cam.R, np.float32).astype(nf))
    t = torch.as_tensor(np.asarray(cam.t, np.float32).astype(nf))
    p = mu @ R.T + t
    fx, fy = float(np.float32(cam.fx)), float(np.float32(cam.fy))
    cx, cy = float(np.float32(cam.cx)), float(np.float32(cam.cy))
    px, py, pz = p[:, 0], p[:, 1], p[:, 2]
    zero = torch.zeros_like(pz)
    # the Jacobian at the laterally clamped point x/z, y/z (3DGS's clamp to
    # 1.3 tan(fov/2), the limits rounded to FP32 as in the oracle's C side)
    limx = float(np.float32(1.3 * (int(W) / (2.0 * float(np.float32(cam.fx))))))
    limy = float(np.float32(1.3 * (int(H) / (2.0 * float(np.float32(cam.fy))))))
    uc = torch.clamp(px / pz, -limx, limx)
    wc = torch.clamp(py / pz, -limy, limy)
    J = torch.stack([torch.stack([fx / pz, zero, -fx * uc / pz], 1),
                     torch.stack([zero, fy / pz, -fy * wc / pz], 1)], 1)
    Tm = J @ R
    C2 = Tm @ Sig @ Tm.transpose(1, 2)
    a = C2[:, 0, 0] + 0.3
    b = C2[:, 0, 1]
    c = C2[:, 1, 1] + 0.3
    det = a * c - b * b
    ca, cb, cc = c / det, -b / det, a / det
    mx = fx * px / pz + cx
    my = fy * py / pz + cy
    center = torch.as_tensor(np.asarray(cam.center, np.float64).astype(nf))
    d = mu - center
    d = d / torch.linalg.norm(d, dim=1, keepdim=True)
    nk = (sh_degree + 1) ** 2
    Y = sh_basis_t(d)[:, :nk]
    rgb = torch.clamp(torch.einsum("nk,nkc->nc", Y, sh[order_t][:, :nk, :]) + 0.5, min=0.0)

    ys, xs = torch.meshgrid(torch.arange(H, dtype=ft) + 0.5,
                            torch.arange(W, dtype=ft) + 0.5, indexing="ij")
    P = torch.stack([xs.reshape(-1), ys.reshape(-1)], 1)
    out = []
    Tfin = []
    ncon = []
    sig = [0.0, 0.0]   # (pairs used, pairs included): fixes the discrete decisions
    for s0 in range(0, P.shape[0], pix_chunk):
        pp = P[s0:s0 + pix_chunk]
        dx = pp[:, :1] - mx[None, :]
        dy = pp[:, 1:] - my[None, :]
        qf = ca[None] * dx * dx + 2 * cb[None] * dx * dy + cc[None] * dy * dy
        alpha = torch.clamp(op[None] * torch.exp(-0.5 * qf), max=0.99)
        with torch.no_grad():
            used = (alpha >= 1.0 / 255.0).to(ft)
            Tinc = torch.cumprod(1.0 - alpha * used, dim=1)
            incl = (Tinc >= 1e-4).to(ft) * used
        sig[0] += float(used.sum())
        sig[1] += float(incl.sum())
        am = alpha * incl
        Texc = torch.cumprod(torch.cat([torch.ones_like(am[:, :1]), 1.0 - am[:, :-1]], 1), dim=1)
        wgt = Texc * am
        out.append(wgt @ rgb)
        if return_aux:
            Tfin.append(torch.prod(1.0 - am, dim=1).detach())
            ncon.append(incl.sum(1).detach())
    img = torch.cat(out, 0).reshape(H, W, 3)
    if return_aux:
        return img, torch.cat(Tfin).reshape(H, W), torch.cat(ncon).reshape(H, W), tuple(sig)
    return img


def params_t(level, requires_grad=True, dtype=torch.float64):
    """Torch copies (FP64 by default) of a synth.Level's raw parameters."""
    nf = np.float64 if dtype == torch.float64 else np.float32

    def t(a):
        x = torch.as_tensor(np.asarray(a, np.float32).astype(nf))
        return x.requires_grad_(requires_grad)
    return (t(level.means), t(level.log_scales), t(level.quats), t(level.opacity_logits), t(level.sh))


def grads(level, cam, weight, sh_degree=3, filter_var=0.0, dtype=torch.float64):
    """Gradients of L = sum(weight * image) w.r.t. (means, log_scales, quats,
    opacity_logits, sh) as numpy arrays.  dtype=torch.float32 evaluates the
    same definition with FP32 rounding: its distance to the FP64 result is
    the error that FP32 arithmetic alone makes on these inputs."""
    ps = params_t(level, dtype=dtype)
    img = render_t(*ps, cam, sh_degree=sh_degree, filter_var=filter_var)
    L = (img * torch.as_tensor(np.asarray(weight, np.float64), dtype=dtype)).sum()
    L.backward()
    return [p.grad.numpy().copy() for p in ps], img.detach().numpy()
