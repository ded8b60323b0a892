"""GPU parity of the particle-bound Gaussians (covariance update, splatting
forward and reverse mode) against the FP64 oracle (oracle/gsplat.py), through
the C-ABI. Pixels where some Gaussian sits within 1e-3 of the q = 9 cut-off
are left out of the element-wise comparison (the in-or-out decision there
depends on rounding) and their number is bounded; the depth order is an
integer decision made on float32 depths, so scenes either have well
separated depths or ties that are exact in any precision."""
import numpy as np
import pytest
import torch

from oracle import gsplat as G
from paper_2603_09668_gb300 import binding as B
from paper_2603_09668_gb300 import inputs

from gpu_util import max_rel, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def cams(cam):
    return (B.camera(cam["R"], cam["T"], cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["width"],
                     cam["height"]),
            G.camera(cam["R"], cam["T"], cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["width"],
                     cam["height"]))


def test_covariance_matches_oracle():
    x, F, s0, _, _, _ = inputs.gaussian_scene(n=1000, seed=3)
    S = B.gs_covariance(to_dev(F), to_dev(s0)).cpu().numpy()
    assert max_rel(S, G.covariance(F, s0)) <= 1e-6


@pytest.mark.parametrize("ties", [False, True])
def test_render_matches_oracle(ties):
    x, F, s0, col, op, cam = inputs.gaussian_scene(n=300, depth_ties=ties, seed=4)
    dcam, ocam = cams(cam)
    W, H = cam["width"], cam["height"]
    r = B.GaussianRenderer(300, W, H)
    img = r.render(dcam, *(to_dev(a) for a in (x, F, s0, col, op))).cpu().numpy()
    ref = G.render(x, F, s0, col, op, ocam)
    edge = G.near_cutoff(x, F, s0, ocam, 1e-3).reshape(H, W)
    assert edge.sum() <= 0.02 * W * H
    keep = ~edge
    assert np.abs(img[:, keep] - ref[:, keep]).max() <= 2e-5
    assert ref.max() > 0.3  # the scene is in view
    r.close()


def test_render_backward_matches_oracle_autograd():
    x, F, s0, col, op, cam = inputs.gaussian_scene(n=120, width=40, height=32, seed=5)
    dcam, ocam = cams(cam)
    W, H = cam["width"], cam["height"]
    g_img = np.random.default_rng(6).standard_normal((3, H, W)).astype(np.float32)
    g_img[:, G.near_cutoff(x, F, s0, ocam, 1e-3).reshape(H, W)] = 0.0
    r = B.GaussianRenderer(120, W, H)
    dx, dF, dc, do = (to_dev(a) for a in (x, F, col, op))
    ds0 = to_dev(s0)
    r.render(dcam, dx, dF, ds0, dc, do)
    g_x, g_F = torch.zeros_like(dx), torch.zeros_like(dF)
    g_c, g_o = torch.zeros_like(dc), torch.zeros_like(do)
    r.backward(dcam, dx, dF, ds0, dc, do, to_dev(g_img), g_x, g_F, g_c, g_o)
    ref = G.render_grad(x, F, s0, col, op, ocam, g_img)
    for name, got in (("x", g_x), ("F", g_F), ("color", g_c), ("opacity", g_o)):
        e = rel_l2(got.cpu().numpy(), ref[name])
        assert e <= 1e-4, (name, e)
    # accumulation: a second backward adds the same again
    r.backward(dcam, dx, dF, ds0, dc, do, to_dev(g_img), g_x, g_F)
    assert rel_l2(g_x.cpu().numpy(), 2 * ref["x"]) <= 1e-4
    r.close()


def test_full_size_render_on_sampled_pixels():
    """100,284 particle-bound Gaussians of the 64^3 sheet at 512 x 512: 200
    sampled pixels against the oracle evaluated at those pixels (the sheet's
    two particle layers tie exactly in depth)."""
    sc = inputs.sheet_scene(nu=274, nv=183, n_grid=64, n_substeps=1, seed=0)
    n = sc.n
    rng = np.random.default_rng(7)
    x = sc.x
    F = np.zeros((9, n), np.float32)
    F[[0, 4, 8]] = 1.0
    F += rng.uniform(-0.05, 0.05, (9, n)).astype(np.float32)
    s0 = np.zeros((6, n), np.float32)
    s0[:3] = 0.003 ** 2
    col = rng.uniform(0, 1, (3, n)).astype(np.float32)
    op = rng.uniform(0.3, 0.9, n).astype(np.float32)
    cam = dict(R=np.eye(3), T=np.array([-0.5, -0.6, 1.2]), fx=600.0, fy=600.0, cx=256.0,
               cy=256.0, width=512, height=512)
    dcam, ocam = cams(cam)
    r = B.GaussianRenderer(n, 512, 512)
    img = r.render(dcam, *(to_dev(a) for a in (x, F, s0, col, op))).cpu().numpy()
    pix = np.stack([rng.integers(150, 362, 200), rng.integers(185, 327, 200)], 1)
    ref = G.render(x, F, s0, col, op, ocam, pixels=pix)
    edge = G.near_cutoff(x, F, s0, ocam, 1e-3, pixels=pix)
    got = img[:, pix[:, 1], pix[:, 0]]
    assert edge.sum() <= 20
    assert np.abs(got[:, ~edge] - ref[:, ~edge]).max() <= 5e-5
    assert ref.max() > 0.3
    r.close()


def test_dssim_matches_oracle():
    rng = np.random.default_rng(9)
    a = rng.random((3, 37, 29)).astype(np.float32)  # no side a multiple of the window
    b = np.clip(a + 0.1 * rng.standard_normal(a.shape), 0, 1).astype(np.float32)
    ref_loss, ref_g = G.dssim_loss(a, b)
    loss = torch.zeros(1, device="cuda")
    g = torch.zeros((3, 37, 29), device="cuda")
    B.image_dssim_loss(to_dev(a), to_dev(b), loss, 0.5, g)
    assert loss.item() == pytest.approx(0.5 * ref_loss, rel=1e-4)
    assert rel_l2(g.cpu().numpy(), 0.5 * ref_g) <= 1e-4
    # identical images: zero loss
    loss.zero_()
    B.image_dssim_loss(to_dev(a), to_dev(a), loss)
    assert abs(loss.item()) < 1e-5


def test_l1_loss_and_edge_cases():
    rng = np.random.default_rng(8)
    a = rng.random((3, 17, 13)).astype(np.float32)
    b = rng.random((3, 17, 13)).astype(np.float32)
    loss = torch.zeros(1, device="cuda")
    g = torch.zeros((3, 17, 13), device="cuda")
    B.image_l1_loss(to_dev(a), to_dev(b), loss, 0.5, g)
    ref_loss, ref_g = G.l1_loss(a, b)
    assert loss.item() == pytest.approx(0.5 * ref_loss * a.size, rel=1e-5)
    assert np.allclose(g.cpu().numpy(), 0.5 * ref_g * a.size, atol=1e-7)
    # no Gaussians: a black image; backward after a render of another count is refused
    cam = B.camera(np.eye(3), (0, 0, 2), 20, 20, 8, 8, 16, 16)
    r = B.GaussianRenderer(4, 16, 16)
    e = torch.zeros((3, 0), device="cuda")
    img = r.render(cam, e, torch.zeros((9, 0), device="cuda"), torch.zeros((6, 0), device="cuda"),
                   e, torch.zeros(0, device="cuda"))
    assert not img.any()
    x = torch.tensor([[0.0], [0.0], [-3.0]], device="cuda")  # t_z = -1: behind the camera
    F = torch.eye(3, device="cuda").reshape(9, 1)
    s0 = torch.tensor([[0.01], [0.01], [0.01], [0.0], [0.0], [0.0]], device="cuda")
    c1, o1 = torch.ones((3, 1), device="cuda"), torch.ones(1, device="cuda")
    with pytest.raises(B.DiffWindError):
        r.backward(cam, x, F, s0, c1, o1, torch.zeros((3, 16, 16), device="cuda"),
                   torch.zeros_like(x), torch.zeros_like(F))
    img = r.render(cam, x, F, s0, c1, o1)
    assert not img.any()
    r.close()
