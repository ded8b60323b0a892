"""Pins for the FP64 surrogate oracle: the direct-sum convolution network
against torch's CPU conv3d in float64 (an independent implementation), its
reverse mode against central differences and against torch autograd, and the
feature / upsample / re-equilibration steps against closed forms."""
import numpy as np
import pytest
import torch
import torch.nn.functional as Fnn

import oracle
from paper_2603_09668_gb300 import inputs

RNG = np.random.default_rng(2024)


def random_params(scale=0.1, seed=0):
    rng = np.random.default_rng(seed)
    p = np.zeros(oracle.surr_num_params())
    for ws, bs, cin, cout in oracle.surr_layer_slices():
        p[ws] = rng.standard_normal(ws.stop - ws.start) * scale / np.sqrt(27 * cin) * 3
        p[bs] = rng.standard_normal(cout) * 0.05
    return p


def torch_forward(n, params, feats):
    x = torch.tensor(feats, dtype=torch.float64).reshape(n, n, n, 16).permute(3, 0, 1, 2)[None]
    for l, (ws, bs, cin, cout) in enumerate(oracle.surr_layer_slices()):
        W = torch.tensor(params[ws]).reshape(3, 3, 3, cout, cin).permute(3, 4, 0, 1, 2)
        b = torch.tensor(params[bs])
        x = Fnn.conv3d(x, W, b, padding=1)
        if l < 3:
            x = 0.5 * x * (1.0 + torch.erf(x / np.sqrt(2.0)))
    return x[0].permute(1, 2, 3, 0).reshape(n ** 3, 16)


@pytest.mark.parametrize("n", [4, 6])
def test_forward_matches_torch_conv3d(n):
    p = random_params(seed=n)
    feats = RNG.standard_normal((n ** 3, 16))
    out = oracle.surr_forward(n, p, feats)
    ref = torch_forward(n, p, feats).numpy()
    assert np.allclose(out, ref, rtol=1e-11, atol=1e-12)


def test_backward_matches_torch_autograd():
    n = 5
    p = random_params(seed=1)
    feats = RNG.standard_normal((n ** 3, 16))
    g_out = RNG.standard_normal((n ** 3, 16))
    g = oracle.surr_backward(n, p, feats, g_out)
    pt = torch.tensor(p, requires_grad=True)
    x = torch.tensor(feats).reshape(n, n, n, 16).permute(3, 0, 1, 2)[None]
    for l, (ws, bs, cin, cout) in enumerate(oracle.surr_layer_slices()):
        W = pt[ws].reshape(3, 3, 3, cout, cin).permute(3, 4, 0, 1, 2)
        x = Fnn.conv3d(x, W, pt[bs], padding=1)
        if l < 3:
            x = 0.5 * x * (1.0 + torch.erf(x / np.sqrt(2.0)))
    out = x[0].permute(1, 2, 3, 0).reshape(n ** 3, 16)
    (out * torch.tensor(g_out)).sum().backward()
    assert np.allclose(g, pt.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_backward_central_differences():
    n = 4
    p = random_params(seed=2)
    feats = RNG.standard_normal((n ** 3, 16))
    g_out = RNG.standard_normal((n ** 3, 16))
    g = oracle.surr_backward(n, p, feats, g_out)
    rng = np.random.default_rng(7)
    for k in rng.choice(p.size, 12, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (np.sum(g_out * oracle.surr_forward(n, pp, feats)) -
              np.sum(g_out * oracle.surr_forward(n, pm, feats))) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_features_closed_forms():
    n = 4
    N = 2 * n
    c, w, _ = oracle.velocity_set()
    # a uniform flow gives rho - 1 = 0 and u everywhere; a full solid coarse
    # voxel gives zero flow features and solid fraction 1
    u0 = np.array([0.04, -0.01, 0.02])
    feq = oracle.lbm_equilibrium(1.02, u0)
    f = np.repeat(feq[:, None], N ** 3, axis=1)
    solid = np.zeros((N, N, N), np.uint8)
    solid[0:2, 0:2, 0:2] = 1       # coarse voxel (0, 0, 0) fully solid
    solid[2, 2, 2] = 1             # one eighth of coarse voxel (1, 1, 1)
    feats, rho, u = oracle.surr_features(n, f, solid.ravel())
    fv = feats.reshape(n, n, n, 16)
    assert np.allclose(fv[0, 0, 0, :4], 0.0) and fv[0, 0, 0, 4] == 1.0
    assert fv[1, 1, 1, 4] == pytest.approx(1 / 8)
    assert np.allclose(fv[2, 3, 1, 0], 0.02) and np.allclose(fv[2, 3, 1, 1:4], u0)
    assert np.all(fv[..., 5:] == 0.0)
    assert np.allclose(rho.reshape(N, N, N)[solid == 0], 1.02)
    # relative to a reference velocity: u - u_ref on voxels with fluid, 0 on a
    # fully solid voxel, u_ref itself in channels 5-7 everywhere
    u_ref = np.array([0.05, 0.01, -0.02])
    feats_r, _, _ = oracle.surr_features(n, f, solid.ravel(), u_ref)
    fr = feats_r.reshape(n, n, n, 16)
    assert np.allclose(fr[2, 3, 1, 1:4], u0 - u_ref) and fr[2, 3, 1, 0] == pytest.approx(0.02)
    assert np.allclose(fr[0, 0, 0, 1:4], 0.0)
    assert np.allclose(fr[..., 5:8], u_ref) and np.all(fr[..., 8:] == 0.0)
    assert np.allclose(fr[..., [0, 4]], fv[..., [0, 4]])


def test_apply_upsampling_and_equilibrium():
    n = 4
    N = 2 * n
    rng = np.random.default_rng(3)
    du = np.zeros((n ** 3, 16))
    du[:, :3] = rng.standard_normal((n ** 3, 3)) * 0.01
    rho = 1.0 + 0.01 * rng.standard_normal(N ** 3)
    u = 0.02 * rng.standard_normal((3, N ** 3))
    c, w, _ = oracle.velocity_set()
    f0 = np.repeat(w[:, None], N ** 3, axis=1)
    f = oracle.surr_apply(n, du, rho, u, f0)
    # upsampled du against torch's trilinear interpolation (align_corners=False)
    dut = torch.tensor(du[:, :3]).reshape(n, n, n, 3).permute(3, 0, 1, 2)[None]
    up = Fnn.interpolate(dut, scale_factor=2, mode="trilinear", align_corners=False)[0]
    up = up.reshape(3, N ** 3).numpy()
    rho_out = f.sum(0)
    mom = c.T @ f
    assert np.allclose(rho_out, rho, atol=1e-14)
    assert np.allclose(mom / rho_out, u + up, atol=1e-13)
    # solid cells keep their populations
    solid = (rng.random(N ** 3) < 0.2).astype(np.uint8)
    f2 = oracle.surr_apply(n, du, rho, u, f0, solid)
    assert np.array_equal(f2[:, solid == 1], f0[:, solid == 1])
