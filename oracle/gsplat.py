"""FP64 oracle of the particle-bound Gaussians: the covariance update under the
deformation gradient (Sec. 3.2, interaction modelling) and the alpha-blended
splatting renderer (Sec. 3.3, Eq. rendering; the 3D Gaussian representation
of the appendix), with its gradient.

TEST INFRASTRUCTURE ONLY: the CUDA path is checked against these functions;
only tests/, the smoke check in __graft_entry__.py and bench.py's reference
leg may import this module. Nothing here is shared with the CUDA library.

Plain float64 torch on the CPU, vectorised over pixels x Gaussians; the
gradient is torch autograd of the same forward (a library primitive), pinned
by central differences in the tests.

Definitions (readings where the paper is silent are marked R):
  - Sigma(t) = F Sigma0 F^T per particle; symmetric 3x3 stored as six values
    (xx, yy, zz, xy, xz, yz); F row-major per particle, F[3a + b] = F_ab.
  - Camera: t = R x + T (camera space, z forward), pinhole projection
    mu' = (fx t_x / t_z + cx, fy t_y / t_z + cy) (the printed mu' = J W mu is
    the affine approximation; R: the exact projection of the centre);
    J = [[fx/t_z, 0, -fx t_x/t_z^2], [0, fy/t_z, -fy t_y/t_z^2]],
    Sigma' = J R Sigma R^T J^T (the printed formula, W = R).
  - A Gaussian takes part only if t_z > near and det Sigma' > 0 (R).
  - alpha_i = o_i exp(-q/2) with q = d^T Sigma'^-1 d, d = pixel centre - mu',
    truncated to 0 beyond three standard deviations, q > 9 (R: the usual
    3-sigma support, written as an exact ellipse so that it is independent
    of any tiling); pixel (px, py) has its centre at (px + 1/2, py + 1/2).
  - C = sum_i T_i c_i alpha_i, T_i = prod_{j<i} (1 - alpha_j), the Gaussians
    in increasing t_z (ties by index); no background term (as printed).
  - Image layout [3][H][W].
  - D-SSIM (the structural term of L_render, Sec. 3.3): 1 - mean over pixels
    and channels of SSIM = ((2 mu_x mu_y + C1)(2 s_xy + C2)) / ((mu_x^2 +
    mu_y^2 + C1)(s_x^2 + s_y^2 + C2)) with the local means and (co)variances
    taken under an 11 x 11 Gaussian window of standard deviation 1.5, zero
    outside the image, C1 = 0.01^2, C2 = 0.03^2 (R: the usual SSIM constants
    and window, which the paper does not restate).
"""
from __future__ import annotations

import numpy as np
import torch

DT = torch.float64


def _sym(s6):
    """[6][n] -> (n, 3, 3)."""
    xx, yy, zz, xy, xz, yz = s6
    row0 = torch.stack([xx, xy, xz], -1)
    row1 = torch.stack([xy, yy, yz], -1)
    row2 = torch.stack([xz, yz, zz], -1)
    return torch.stack([row0, row1, row2], -2)


def _six(S):
    """(n, 3, 3) -> [6][n]."""
    return torch.stack([S[:, 0, 0], S[:, 1, 1], S[:, 2, 2], S[:, 0, 1], S[:, 0, 2], S[:, 1, 2]])


def covariance(F, sigma0):
    """Sigma = F Sigma0 F^T for F [9][n] and sigma0 [6][n]; returns [6][n]."""
    F = torch.as_tensor(np.asarray(F, np.float64))
    n = F.shape[1]
    Fm = F.T.reshape(n, 3, 3)
    S = Fm @ _sym(torch.as_tensor(np.asarray(sigma0, np.float64))) @ Fm.transpose(1, 2)
    return _six(S).numpy()


def camera(R, T, fx, fy, cx, cy, width, height, near=0.01):
    return dict(R=np.asarray(R, np.float64).reshape(3, 3), T=np.asarray(T, np.float64).reshape(3),
                fx=float(fx), fy=float(fy), cx=float(cx), cy=float(cy), width=int(width),
                height=int(height), near=float(near))


def _render(x, F, s0, color, opacity, cam, pixels=None, want_q=False):
    n = x.shape[1]
    R = torch.as_tensor(cam["R"], dtype=DT)
    T = torch.as_tensor(cam["T"], dtype=DT)
    fx, fy, cx, cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    W, H = cam["width"], cam["height"]
    Fm = F.T.reshape(n, 3, 3)
    Sig = Fm @ _sym(s0) @ Fm.transpose(1, 2)
    t = x.T @ R.T + T
    tx, ty, tz = t[:, 0], t[:, 1], t[:, 2]
    vis = (tz > cam["near"]).detach()
    tzs = torch.where(vis, tz, torch.ones_like(tz))  # keep the arithmetic finite where unused
    J = torch.zeros(n, 2, 3, dtype=DT)
    J[:, 0, 0] = fx / tzs
    J[:, 0, 2] = -fx * tx / tzs ** 2
    J[:, 1, 1] = fy / tzs
    J[:, 1, 2] = -fy * ty / tzs ** 2
    S2 = J @ R @ Sig @ R.T @ J.transpose(1, 2)
    det = S2[:, 0, 0] * S2[:, 1, 1] - S2[:, 0, 1] * S2[:, 1, 0]
    vis = vis & (det > 0).detach()
    dets = torch.where(vis, det, torch.ones_like(det))
    ca = S2[:, 1, 1] / dets
    cb = -S2[:, 0, 1] / dets
    cc = S2[:, 0, 0] / dets
    mux = fx * tx / tzs + cx
    muy = fy * ty / tzs + cy
    if pixels is None:
        py, px = torch.meshgrid(torch.arange(H, dtype=DT) + 0.5, torch.arange(W, dtype=DT) + 0.5,
                                indexing="ij")
    else:
        pix = torch.as_tensor(np.asarray(pixels), dtype=DT)
        px, py = pix[:, 0] + 0.5, pix[:, 1] + 0.5
    dx = px.reshape(-1, 1) - mux.reshape(1, -1)
    dy = py.reshape(-1, 1) - muy.reshape(1, -1)
    q = ca * dx * dx + 2 * cb * dx * dy + cc * dy * dy
    if want_q:
        return torch.where(vis.reshape(1, -1), q, torch.full_like(q, float("inf")))
    inside = ((q <= 9.0) & vis.reshape(1, -1)).detach()
    alpha = torch.where(inside, opacity.reshape(1, -1) * torch.exp(-0.5 * q),
                        torch.zeros_like(q))
    order = np.lexsort((np.arange(n), tz.detach().numpy()))  # by depth, ties by index
    order = torch.as_tensor(order, dtype=torch.long)
    a = alpha[:, order]
    trans = torch.cumprod(torch.cat([torch.ones(a.shape[0], 1, dtype=DT), 1 - a[:, :-1]], 1), 1)
    wgt = trans * a  # (HW, n)
    img = wgt @ color.T[order]  # (HW, 3)
    return img.T.reshape(3, H, W) if pixels is None else img.T


def _tensors(x, F, sigma0, color, opacity, grad=False):
    return [torch.tensor(np.ascontiguousarray(a, np.float64), dtype=DT, requires_grad=grad)
            for a in (x, F, sigma0, color, opacity)]


def render(x, F, sigma0, color, opacity, cam, pixels=None):
    """Image [3][H][W] of Gaussians at x [3][n] with F [9][n], rest
    covariances sigma0 [6][n], colours [3][n] and opacities [n]; or, with
    pixels (m, 2) integer (px, py), the colours [3][m] of those pixels."""
    with torch.no_grad():
        return _render(*_tensors(x, F, sigma0, color, opacity), cam, pixels).numpy()


def near_cutoff(x, F, sigma0, cam, tol, pixels=None):
    """Mask ([H*W] or [m]) of the pixels where some drawn Gaussian has its
    Mahalanobis q within tol of the cut-off 9: there the in-or-out decision
    depends on rounding, so a float32 renderer may decide otherwise."""
    n = np.asarray(x).shape[1]
    t = _tensors(x, F, sigma0, np.zeros((3, n)), np.zeros(n))
    with torch.no_grad():
        q = _render(*t, cam, pixels, want_q=True)
    return (torch.abs(q - 9.0) < tol).any(dim=1).numpy()


def render_grad(x, F, sigma0, color, opacity, cam, g_image):
    """Gradients of sum(g_image * image) with respect to x, F, color, opacity."""
    tx, tF, ts, tc, to = _tensors(x, F, sigma0, color, opacity, grad=True)
    img = _render(tx, tF, ts, tc, to, cam)
    (img * torch.as_tensor(np.asarray(g_image, np.float64))).sum().backward()
    return dict(x=tx.grad.numpy(), F=tF.grad.numpy(), color=tc.grad.numpy(),
                opacity=to.grad.numpy())


def l1_loss(image, target):
    """(mean |image - target|, its gradient) over all values."""
    d = np.asarray(image, np.float64) - np.asarray(target, np.float64)
    return float(np.mean(np.abs(d))), np.sign(d) / d.size


SSIM_C1, SSIM_C2 = 0.01 ** 2, 0.03 ** 2


def _ssim_window():
    k = torch.exp(-((torch.arange(11, dtype=DT) - 5.0) ** 2) / (2 * 1.5 ** 2))
    k = k / k.sum()
    return torch.outer(k, k)


def _dssim(img, tgt):
    """img, tgt (C, H, W) float64 tensors -> 1 - mean SSIM."""
    C = img.shape[0]
    w = _ssim_window().expand(C, 1, 11, 11).contiguous()
    blur = lambda a: torch.nn.functional.conv2d(a[None], w, padding=5, groups=C)[0]
    mx, my = blur(img), blur(tgt)
    sxx = blur(img * img) - mx * mx
    syy = blur(tgt * tgt) - my * my
    sxy = blur(img * tgt) - mx * my
    ssim = ((2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)) / (
        (mx * mx + my * my + SSIM_C1) * (sxx + syy + SSIM_C2))
    return 1.0 - ssim.mean()


def dssim_loss(image, target):
    """(1 - mean SSIM, its gradient with respect to image) for [C][H][W]."""
    img = torch.tensor(np.ascontiguousarray(image, np.float64), requires_grad=True)
    tgt = torch.tensor(np.ascontiguousarray(target, np.float64))
    d = _dssim(img, tgt)
    d.backward()
    return float(d.detach()), img.grad.numpy()
