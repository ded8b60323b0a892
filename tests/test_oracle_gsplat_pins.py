"""Pins of the Gaussian oracle (oracle/gsplat.py) against closed forms: the
covariance update under rotations, scalings and the identity; one isotropic
Gaussian on the optical axis renders the textbook 2D Gaussian of width
f sigma / z, truncated at three standard deviations; a point off the axis
lands at the pinhole projection; two Gaussians composite front to back
whatever order they are given in; the L1 term; the gradient by central
differences."""
import numpy as np
import pytest

from oracle import gsplat as G


def eye9(n):
    F = np.zeros((9, n))
    F[[0, 4, 8]] = 1.0
    return F


def iso6(n, s2):
    s = np.zeros((6, n))
    s[:3] = s2
    return s


def rot(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def full(s6):
    xx, yy, zz, xy, xz, yz = s6
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def test_covariance_update_closed_forms():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((3, 3))
    S0 = A @ A.T + 0.1 * np.eye(3)
    s0 = np.array([S0[0, 0], S0[1, 1], S0[2, 2], S0[0, 1], S0[0, 2], S0[1, 2]])[:, None]
    Rm = rot((1, 2, 3), 0.7)
    S = full(G.covariance(Rm.reshape(9, 1), s0)[:, 0])
    assert np.allclose(S, Rm @ S0 @ Rm.T, atol=1e-14)
    assert np.allclose(np.linalg.eigvalsh(S), np.linalg.eigvalsh(S0), atol=1e-13)
    S = full(G.covariance((1.7 * np.eye(3)).reshape(9, 1), s0)[:, 0])
    assert np.allclose(S, 1.7 ** 2 * S0, atol=1e-14)
    assert np.allclose(G.covariance(eye9(1), s0), s0, atol=0)


def test_single_gaussian_on_axis_is_the_2d_gaussian():
    W, H, f, z, sig = 40, 30, 50.0, 2.0, 0.1
    cam = G.camera(np.eye(3), np.zeros(3), f, f, W / 2, H / 2, W, H)
    x = np.array([[0.0], [0.0], [z]])
    img = G.render(x, eye9(1), iso6(1, sig ** 2), np.array([[0.9], [0.5], [0.2]]),
                   np.array([0.8]), cam)
    s = f * sig / z  # 2.5 pixels
    py, px = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    r2 = (px - W / 2) ** 2 + (py - H / 2) ** 2
    expect = np.where(r2 <= 9 * s * s, 0.8 * np.exp(-0.5 * r2 / (s * s)), 0.0)
    for ch, c in enumerate((0.9, 0.5, 0.2)):
        assert np.allclose(img[ch], c * expect, atol=1e-14)


def test_off_axis_centre_is_the_pinhole_projection():
    W, H, f = 64, 48, 40.0
    Rm = rot((0, 1, 0), 0.2)
    T = np.array([0.1, -0.2, 3.0])
    cam = G.camera(Rm, T, f, 1.1 * f, 31.0, 22.0, W, H)
    X = np.array([0.3, 0.2, -0.4])
    t = Rm @ X + T
    u, v = f * t[0] / t[2] + 31.0, 1.1 * f * t[1] / t[2] + 22.0
    # the intensity centroid of a Gaussian about 2 pixels wide is its projected centre
    img = G.render(X[:, None], eye9(1), iso6(1, 0.15 ** 2), np.ones((3, 1)), np.array([0.5]), cam)
    py, px = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    w = img[0] / img[0].sum()
    assert np.sum(w * px) == pytest.approx(u, abs=0.02)
    assert np.sum(w * py) == pytest.approx(v, abs=0.02)


def test_two_gaussians_composite_front_to_back():
    W, H, f = 9, 9, 30.0
    cam = G.camera(np.eye(3), np.zeros(3), f, f, 4.5, 4.5, W, H)
    x = np.array([[0.0, 0.0], [0.0, 0.0], [2.0, 3.0]])
    col = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    op = np.array([0.6, 0.7])
    s0 = iso6(2, 0.05 ** 2)
    img = G.render(x, eye9(2), s0, col, op, cam)
    # centre pixel: alpha = opacity; the nearer (z = 2) is composited first
    assert img[0, 4, 4] == pytest.approx(0.6, abs=1e-14)
    assert img[1, 4, 4] == pytest.approx((1 - 0.6) * 0.7, abs=1e-14)
    swapped = G.render(x[:, ::-1], eye9(2), s0, col[:, ::-1], op[::-1], cam)
    assert np.allclose(img, swapped, atol=1e-15)
    # behind the camera: no contribution
    back = G.render(np.array([[0.0], [0.0], [-2.0]]), eye9(1), iso6(1, 0.01), np.ones((3, 1)),
                    np.array([0.9]), cam)
    assert not back.any()


def test_pixel_subset_matches_the_full_image():
    rng = np.random.default_rng(2)
    n, W, H = 7, 20, 14
    cam = G.camera(np.eye(3), np.array([0.0, 0.0, 2.0]), 25.0, 25.0, 10, 7, W, H)
    x = rng.uniform(-0.3, 0.3, (3, n))
    s0 = iso6(n, 0.06 ** 2)
    col, op = rng.uniform(0, 1, (3, n)), rng.uniform(0.2, 0.9, n)
    img = G.render(x, eye9(n), s0, col, op, cam)
    pix = np.stack([rng.integers(0, W, 30), rng.integers(0, H, 30)], 1)
    sub = G.render(x, eye9(n), s0, col, op, cam, pixels=pix)
    assert np.allclose(sub, img[:, pix[:, 1], pix[:, 0]], atol=1e-15)


def test_dssim_identical_images_and_brute_force():
    rng = np.random.default_rng(3)
    a = rng.random((2, 13, 17))
    d, g = G.dssim_loss(a, a)
    assert d == pytest.approx(0.0, abs=1e-12)
    assert np.abs(g).max() < 1e-12  # a minimum
    # brute force on a tiny image: window sums written out pixel by pixel
    b = rng.random((1, 7, 6))
    c = rng.random((1, 7, 6))
    k1 = np.exp(-((np.arange(11) - 5.0) ** 2) / (2 * 1.5 ** 2))
    k1 /= k1.sum()
    H, W = 7, 6
    tot = 0.0
    for yy in range(H):
        for xx in range(W):
            m = {"x": 0.0, "y": 0.0, "xx": 0.0, "yy": 0.0, "xy": 0.0}
            for dy in range(-5, 6):
                for dx in range(-5, 6):
                    py_, px_ = yy + dy, xx + dx
                    if 0 <= py_ < H and 0 <= px_ < W:
                        wgt = k1[dy + 5] * k1[dx + 5]
                        u, v = b[0, py_, px_], c[0, py_, px_]
                        m["x"] += wgt * u
                        m["y"] += wgt * v
                        m["xx"] += wgt * u * u
                        m["yy"] += wgt * v * v
                        m["xy"] += wgt * u * v
            sx = m["xx"] - m["x"] ** 2
            sy = m["yy"] - m["y"] ** 2
            sxy = m["xy"] - m["x"] * m["y"]
            c1, c2 = 0.01 ** 2, 0.03 ** 2
            tot += ((2 * m["x"] * m["y"] + c1) * (2 * sxy + c2)) / (
                (m["x"] ** 2 + m["y"] ** 2 + c1) * (sx + sy + c2))
    assert G.dssim_loss(b, c)[0] == pytest.approx(1.0 - tot / (H * W), abs=1e-12)


def test_dssim_gradient_by_central_differences():
    rng = np.random.default_rng(4)
    a, b = rng.random((3, 9, 8)), rng.random((3, 9, 8))
    _, g = G.dssim_loss(a, b)
    eps = 1e-6
    for k in rng.choice(a.size, 10, replace=False):
        p_, m_ = a.copy(), a.copy()
        p_.reshape(-1)[k] += eps
        m_.reshape(-1)[k] -= eps
        fd = (G.dssim_loss(p_, b)[0] - G.dssim_loss(m_, b)[0]) / (2 * eps)
        assert g.reshape(-1)[k] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_l1_loss():
    a = np.array([[0.5, 0.25], [1.0, 0.0]])
    b = np.array([[0.0, 0.5], [1.0, 0.5]])
    loss, g = G.l1_loss(a, b)
    assert loss == pytest.approx((0.5 + 0.25 + 0 + 0.5) / 4)
    assert np.allclose(g, np.array([[1, -1], [0, -1]]) / 4)


def test_gradient_by_central_differences():
    rng = np.random.default_rng(1)
    n, W, H, f = 6, 16, 12, 20.0
    cam = G.camera(rot((0.3, 1, 0.2), 0.25), np.array([0.0, 0.0, 2.5]), f, f, 8, 6, W, H)
    x = rng.uniform(-0.3, 0.3, (3, n))
    F = eye9(n) + 0.1 * rng.standard_normal((9, n))
    s0 = iso6(n, 0.08 ** 2)
    s0[3:] = 0.2 * 0.08 ** 2 * rng.uniform(-1, 1, (3, n))
    col = rng.uniform(0, 1, (3, n))
    op = rng.uniform(0.3, 0.9, n)
    g_img = rng.standard_normal((3, H, W))
    grads = G.render_grad(x, F, s0, col, op, cam, g_img)

    def L(x_, F_, c_, o_):
        return float(np.sum(g_img * G.render(x_, F_, s0, c_, o_, cam)))

    eps = 1e-6
    for name, arr in (("x", x), ("F", F), ("color", col), ("opacity", op)):
        flat = arr.reshape(-1)
        for k in rng.choice(flat.size, size=min(8, flat.size), replace=False):
            args = {"x": x, "F": F, "color": col, "opacity": op}
            p, m = arr.copy(), arr.copy()
            p.reshape(-1)[k] += eps
            m.reshape(-1)[k] -= eps
            ap, am = dict(args), dict(args)
            ap[name], am[name] = p, m
            fd = (L(ap["x"], ap["F"], ap["color"], ap["opacity"]) -
                  L(am["x"], am["F"], am["color"], am["opacity"])) / (2 * eps)
            assert grads[name].reshape(-1)[k] == pytest.approx(fd, rel=1e-5, abs=1e-8), (name, k)


def test_off_axis_shape_is_the_projected_covariance():
    """An isotropic Gaussian off the axis projects to sigma^2 J J^T, J the
    Jacobian of the pinhole projection at its centre (taken here by central
    differences of the projection itself). The image's intensity covariance
    equals that times the variance factor of a 2D Gaussian cut at Mahalanobis
    radius 3, (1 - 5.5 e^-4.5) / (1 - e^-4.5)."""
    W, H, f = 96, 96, 120.0
    cam = G.camera(np.eye(3), np.zeros(3), f, f, 48.0, 48.0, W, H)
    X = np.array([0.55, -0.4, 1.6])  # well off the axis: J couples z into x and y
    sig = 0.03
    img = G.render(X[:, None], eye9(1), iso6(1, sig ** 2), np.ones((3, 1)), np.array([0.5]), cam)

    def proj(t):
        return np.array([f * t[0] / t[2] + 48.0, f * t[1] / t[2] + 48.0])

    J = np.zeros((2, 3))
    for a in range(3):
        e = np.zeros(3)
        e[a] = 1e-6
        J[:, a] = (proj(X + e) - proj(X - e)) / 2e-6
    S2 = sig ** 2 * J @ J.T
    py, px = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    w = img[0] / img[0].sum()
    mx, my = np.sum(w * px), np.sum(w * py)
    cov = np.array([[np.sum(w * (px - mx) ** 2), np.sum(w * (px - mx) * (py - my))],
                    [np.sum(w * (px - mx) * (py - my)), np.sum(w * (py - my) ** 2)]])
    k = (1 - 5.5 * np.exp(-4.5)) / (1 - np.exp(-4.5))
    assert np.allclose(cov, k * S2, rtol=0.02, atol=0.02 * np.abs(S2).max())
