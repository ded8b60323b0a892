"""Pins for the FP64 MPM oracle against what the method and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, invariants, textbook definitions evaluated by brute force, and central
finite differences of the forward. A dropped term, a wrong sign, a wrong
stencil offset or a transposed operand in the oracle fails at least one test.
"""
import numpy as np
import pytest

import oracle
from paper_2603_09668_gb300 import inputs

RNG = np.random.default_rng(1234)


def bspline(r):
    """Textbook quadratic B-spline kernel N(r) (the MLS-MPM kernel, App. A.3)."""
    r = np.abs(r)
    return np.where(r < 0.5, 0.75 - r * r, np.where(r < 1.5, 0.5 * (1.5 - r) ** 2, 0.0))


# ---------------------------------------------------------------- weights --

@pytest.mark.parametrize("fx", list(RNG.uniform(0.5, 1.5, 25)) + [0.5, 1.0, 1.4999999])
def test_bspline_partition_linear_quadratic_moments(fx):
    w = oracle.bspline_weights(fx)
    o = np.arange(3) - fx
    assert abs(w.sum() - 1.0) < 1e-14                      # partition of unity
    assert abs((w * o).sum()) < 1e-14                      # linear reproduction
    assert abs((w * o * o).sum() - 0.25) < 1e-14           # second moment dx^2/4 -> D = 4/dx^2
    assert np.allclose(w, bspline(o), atol=1e-15)          # the textbook kernel


# ----------------------------------------------------------- constitutive --

def test_lame_closed_form():
    mu, lam = oracle.lame(1e4, 0.3)
    assert mu == pytest.approx(1e4 / 2.6, rel=1e-15)
    assert lam == pytest.approx(1e4 * 0.3 / (1.3 * 0.4), rel=1e-15)


def random_F(scale, rng=RNG):
    F = np.eye(3) + rng.uniform(-scale, scale, (3, 3))
    assert np.linalg.det(F) > 0
    return F


@pytest.mark.parametrize("material", [0, 1])
def test_stress_vanishes_at_rest(material):
    assert np.abs(oracle.stress(material, np.eye(3), 5e4, 0.3)).max() < 1e-10


@pytest.mark.parametrize("material", [0, 1])
@pytest.mark.parametrize("scale", [0.05, 0.3])
def test_stress_is_energy_gradient(material, scale):
    """P = dpsi/dF by central differences of the energy (Eq. constitutive_model
    for Neo-Hookean; mu|F-R|^2 + lam/2 (J-1)^2 for fixed-corotated)."""
    E, nu = 5e4, 0.3
    for _ in range(4):
        F = random_F(scale)
        P = oracle.stress(material, F, E, nu)
        h = 1e-6
        Pfd = np.zeros((3, 3))
        for a in range(3):
            for b in range(3):
                Fp, Fm = F.copy(), F.copy()
                Fp[a, b] += h
                Fm[a, b] -= h
                Pfd[a, b] = (oracle.psi(material, Fp, E, nu) - oracle.psi(material, Fm, E, nu)) / (2 * h)
        assert np.abs(P - Pfd).max() <= 1e-6 * max(1.0, np.abs(P).max())


def test_neohookean_matches_textbook_form():
    """mu (F - F^-T) + lam ln J F^-T, evaluated with numpy's inverse."""
    F = random_F(0.2)
    mu, lam = oracle.lame(4e5, 0.3)
    FinvT = np.linalg.inv(F).T
    P = mu * (F - FinvT) + lam * np.log(np.linalg.det(F)) * FinvT
    assert np.allclose(oracle.stress(0, F, 4e5, 0.3), P, rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("scale", [0.05, 0.4])
def test_polar_decomposition_properties(scale):
    for _ in range(5):
        F = random_F(scale)
        R, S = oracle.polar(F)
        assert np.allclose(R.T @ R, np.eye(3), atol=1e-13)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-13)
        assert np.allclose(S, S.T, atol=1e-12)
        assert np.all(np.linalg.eigvalsh(0.5 * (S + S.T)) > 0)
        assert np.allclose(R @ S, F, atol=1e-13)
        # the same factor from numpy's SVD: R = U V^T
        U, _, Vt = np.linalg.svd(F)
        assert np.allclose(R, U @ Vt, atol=1e-12)


@pytest.mark.parametrize("material", [0, 1])
def test_stress_adjoint_finite_differences(material):
    E, nu = 1e4, 0.3
    for _ in range(4):
        F = random_F(0.25)
        Pbar = RNG.standard_normal((3, 3))
        Fbar = oracle.stress_adjoint(material, F, E, nu, Pbar)
        h = 1e-6
        fd = np.zeros((3, 3))
        for a in range(3):
            for b in range(3):
                Fp, Fm = F.copy(), F.copy()
                Fp[a, b] += h
                Fm[a, b] -= h
                fd[a, b] = (np.sum(Pbar * oracle.stress(material, Fp, E, nu))
                            - np.sum(Pbar * oracle.stress(material, Fm, E, nu))) / (2 * h)
        assert np.abs(Fbar - fd).max() <= 1e-6 * np.abs(fd).max()


# ------------------------------------------------------------------- wind --

def test_wind_constant_and_affine_fields_are_reproduced():
    nf, nt, T = 5, 4, 0.3
    grid = np.linspace(0, 1, nf)
    Z, Y, X = np.meshgrid(grid, grid, grid, indexing="ij")
    times = np.linspace(0, T, nt)
    vals = np.zeros((nt, nf, nf, nf, 3))
    coef = RNG.standard_normal((3, 5))
    for f in range(nt):
        for c in range(3):
            vals[f, ..., c] = coef[c, 0] + coef[c, 1] * X + coef[c, 2] * Y + coef[c, 3] * Z + coef[c, 4] * times[f]
    pos = RNG.uniform(0, 1, (3, 50))
    for t in [0.0, 0.05, 0.1499, 0.3, 0.2222]:
        out = oracle.wind_sample(vals, nf, nt, T, pos, t)
        expect = coef[:, :1] + coef[:, 1:2] * pos[0] + coef[:, 2:3] * pos[1] + coef[:, 3:4] * pos[2] + coef[:, 4:5] * t
        assert np.allclose(out, expect, atol=1e-12)
    # a multilinear product x*y*z*t is reproduced exactly too
    prod = np.stack([X * Y * Z * tt for tt in times])[..., None].repeat(3, -1)
    out = oracle.wind_sample(prod, nf, nt, T, pos, 0.1)
    # only exact at nodes in space; between nodes trilinear of x*y*z equals x*y*z
    assert np.allclose(out[0], pos[0] * pos[1] * pos[2] * 0.1, atol=1e-12)
    # clamping outside the unit cube and outside [0, T]
    out_lo = oracle.wind_sample(vals, nf, nt, T, np.full((3, 1), -0.5), -1.0)
    assert np.allclose(out_lo[:, 0], vals[0, 0, 0, 0], atol=1e-12)
    out_hi = oracle.wind_sample(vals, nf, nt, T, np.full((3, 1), 1.5), 9.0)
    assert np.allclose(out_hi[:, 0], vals[-1, -1, -1, -1], atol=1e-12)


def test_wind_single_frame_and_node_values():
    vals = inputs.fourier_wind(6, 1, seed=3).astype(np.float64)
    nodes = np.array([[0.2, 0.4, 0.6], [1.0, 0.0, 0.8], [0.0, 0.0, 0.0]])  # node coords
    out = oracle.wind_sample(vals, 6, 1, 1.0, nodes, 0.77)
    for k in range(3):
        i, j, l = (np.round(nodes[:, k] * 5)).astype(int)
        assert np.allclose(out[:, k], vals[0, l, j, i], atol=1e-12)


def test_wind_adjoint_dot_product():
    nf, nt, T = 4, 3, 1.0
    vals = RNG.standard_normal((nt, nf, nf, nf, 3))
    pos = RNG.uniform(-0.1, 1.1, (3, 40))
    g = RNG.standard_normal((3, 40))
    a = RNG.standard_normal(vals.shape)
    for t in [0.1, 0.5, 0.99]:
        lhs = np.sum(oracle.wind_sample(a, nf, nt, T, pos, t) * g)
        rhs = np.sum(a * oracle.wind_sample_adjoint(vals, nf, nt, T, pos, t, g))
        assert lhs == pytest.approx(rhs, rel=1e-12)


# -------------------------------------------------------------------- P2G --

def small_scene(n=60, N=12, material=1, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.3, 0.7, (3, n))
    v = rng.uniform(-1, 1, (3, n))
    C = rng.uniform(-3, 3, (9, n))
    F = (np.eye(3).reshape(9, 1) + rng.uniform(-0.1, 0.1, (9, n)))
    params = dict(n_grid=N, dt=1e-3, gravity=(0.0, -9.8, 0.0), bc_band=2, material=material,
                  E=2e3, nu=0.3, p_mass=0.01, p_vol=1e-5)
    return params, (x, v, C, F)


@pytest.mark.parametrize("material", [0, 1])
def test_p2g_conserves_mass_and_momentum(material):
    params, (x, v, C, F) = small_scene(material=material)
    gm, gp = oracle.mpm_p2g(params, x, v, C, F)
    m = params["p_mass"]
    assert gm.sum() == pytest.approx(m * x.shape[1], rel=1e-13)
    assert np.allclose(gp.sum(axis=1), m * v.sum(axis=1), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("material", [0, 1])
def test_p2g_brute_force_over_all_nodes(material):
    """Every node of a small grid against the kernel N((x_i - x_p)/dx)."""
    params, (x, v, C, F) = small_scene(n=3, N=8, material=material, seed=5)
    N = params["n_grid"]
    dx = 1.0 / N
    gm, gp = oracle.mpm_p2g(params, x, v, C, F)
    idx = np.arange(N)
    K, J, I = np.meshgrid(idx, idx, idx, indexing="ij")
    xi = np.stack([I.ravel(), J.ravel(), K.ravel()]) * dx
    m = params["p_mass"]
    kappa = params["dt"] * params["p_vol"] * 4.0 / dx ** 2
    bm = np.zeros(N ** 3)
    bp = np.zeros((3, N ** 3))
    for p in range(x.shape[1]):
        d = xi - x[:, p:p + 1]
        W = bspline(d[0] / dx) * bspline(d[1] / dx) * bspline(d[2] / dx)
        Fp = F[:, p].reshape(3, 3)
        P = oracle.stress(material, Fp, params["E"], params["nu"])
        A = -kappa * P @ Fp.T + m * C[:, p].reshape(3, 3)
        bm += W * m
        bp += W * (m * v[:, p:p + 1] + A @ d)
    assert np.allclose(gm, bm, rtol=1e-12, atol=1e-16)
    assert np.allclose(gp, bp, rtol=1e-11, atol=1e-14)


def test_grid_update_stage_against_the_formula():
    """The grid-update stage (mpm_grid_update) on every node of a 12^3 grid:
    v_i = p_i / m_i + dt (g + a_w(x_i, t)) where m_i > 0 outside the sticky
    band, else 0, with the wind sampled by the (separately pinned) sampler."""
    params, _ = small_scene(N=12)
    N, dt, band = params["n_grid"], params["dt"], params["bc_band"]
    rng = np.random.default_rng(21)
    gm = np.where(rng.random(N ** 3) < 0.6, rng.uniform(0.1, 2.0, N ** 3), 0.0)
    gp = rng.standard_normal((3, N ** 3))
    wind = (inputs.fourier_wind(4, 3, seed=2), 4, 3, 0.05)
    t = 0.017
    gv = oracle.mpm_grid_update(params, gm, gp, wind, t)
    idx = np.arange(N)
    K, J, I = np.meshgrid(idx, idx, idx, indexing="ij")
    ijk = np.stack([I.ravel(), J.ravel(), K.ravel()])
    a = oracle.wind_sample(*wind, ijk / N, t)
    inner = np.all((ijk >= band) & (ijk <= N - 1 - band), axis=0)
    live = inner & (gm > 0)
    ref = np.zeros((3, N ** 3))
    g = np.asarray(params["gravity"])[:, None]
    ref[:, live] = gp[:, live] / gm[live] + dt * (g + a[:, live])
    assert live.sum() > 50 and (~live & (gm > 0)).sum() > 50
    assert np.allclose(gv, ref, rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("pinned", [False, True])
def test_g2p_stage_brute_force_over_all_nodes(pinned):
    """The G2P stage (mpm_g2p) against Eqs. G2P and deformation_update summed
    over every node of an 8^3 grid with the kernel N((x_i - x_p)/dx):
    v_p = sum w v_i, C_p = (4/dx^2) sum w v_i (x_i - x_p)^T, x_p + dt v_p,
    (I + dt C_p) F_p; a pinned particle keeps v = C = 0."""
    params, (x, _, _, F) = small_scene(n=5, N=8, seed=9)
    N, dt = params["n_grid"], params["dt"]
    dx = 1.0 / N
    gv = np.random.default_rng(3).standard_normal((3, N ** 3))
    pin = np.zeros(x.shape[1], np.uint8)
    if pinned:
        pin[[1, 3]] = 1
    xo, vo, Co, Fo = oracle.mpm_g2p(params, x, F, gv, pin)
    idx = np.arange(N)
    K, J, I = np.meshgrid(idx, idx, idx, indexing="ij")
    xi = np.stack([I.ravel(), J.ravel(), K.ravel()]) * dx
    for p in range(x.shape[1]):
        d = xi - x[:, p:p + 1]
        W = bspline(d[0] / dx) * bspline(d[1] / dx) * bspline(d[2] / dx)
        v = (W * gv).sum(axis=1)
        Cm = 4.0 / dx ** 2 * (W * gv) @ d.T
        if pin[p]:
            v, Cm = np.zeros(3), np.zeros((3, 3))
        assert np.allclose(vo[:, p], v, rtol=1e-12, atol=1e-14)
        assert np.allclose(Co[:, p], Cm.ravel(), rtol=1e-11, atol=1e-12)
        assert np.allclose(xo[:, p], x[:, p] + dt * v, rtol=1e-14, atol=1e-15)
        Fn = (np.eye(3) + dt * Cm) @ F[:, p].reshape(3, 3)
        assert np.allclose(Fo[:, p], Fn.ravel(), rtol=1e-13, atol=1e-14)


# ---------------------------------------------------------------- substep --

@pytest.mark.parametrize("material", [0, 1])
def test_rigid_translation_is_exact(material):
    """F = I, C = 0, uniform v, no gravity or wind: v stays, x moves by n dt v."""
    x = inputs.block_particles(sub=6, per_sub=1).astype(np.float64)
    n = x.shape[1]
    v0 = np.array([0.3, -0.2, 0.1])
    state = (x, np.tile(v0[:, None], (1, n)), np.zeros((9, n)), np.tile(np.eye(3).reshape(9, 1), (1, n)))
    params = dict(n_grid=32, dt=1e-3, gravity=(0.0, 0.0, 0.0), bc_band=3, material=material,
                  E=1e4, nu=0.3, p_mass=1e-3, p_vol=1e-6)
    wind = (np.zeros((1, 2, 2, 2, 3)), 2, 1, 1.0)
    s = oracle.mpm_rollout(params, state, wind, 0.0, 10)
    assert np.allclose(s[1], v0[:, None], atol=1e-12)
    assert np.abs(s[2]).max() < 1e-10
    assert np.allclose(s[3], np.eye(3).reshape(9, 1), atol=1e-12)
    assert np.allclose(s[0], x + 10 * 1e-3 * v0[:, None], atol=1e-13)


@pytest.mark.parametrize("material", [0, 1])
def test_uniform_acceleration_closed_form(material):
    """The block scene (constant 5 N/kg wind, gravity, no wall contact): an
    undeformed block stays rigid, x_n = x_0 + dt^2 a n(n+1)/2 with a = g + a_w."""
    sc = inputs.block_scene()
    sc.material = material
    x = sc.x.astype(np.float64)
    state = inputs.rest_state(sc.x)
    state = tuple(a.astype(np.float64) for a in state)
    n_sub = 100
    s = oracle.mpm_rollout(sc.params(), state, sc.wind_tuple(), 0.0, n_sub)
    a = np.array([5.0, -9.8, 0.0])
    expect = x + sc.dt ** 2 * a[:, None] * n_sub * (n_sub + 1) / 2
    assert np.abs(s[0] - expect).max() < 1e-12
    assert np.allclose(s[1], (n_sub * sc.dt * a)[:, None], atol=1e-12)
    assert np.allclose(s[3], np.eye(3).reshape(9, 1), atol=1e-12)
    # the closed-form displacement after 100 substeps: 2.525e-4 in x, -4.949e-4 in y
    assert (expect - x)[0, 0] == pytest.approx(2.525e-4, rel=1e-12)
    assert (expect - x)[1, 0] == pytest.approx(-4.9490e-4, rel=1e-12)


def test_rigid_rotation_preserved_by_affine_transfer():
    """v = w x (x - xc), C = skew(w), F = I: one substep keeps v_p = w x (x_p - xc)
    and C_p = skew(w) exactly (APIC + quadratic B-spline; fixes D = 4/dx^2)."""
    x = inputs.block_particles(sub=5, per_sub=1).astype(np.float64)
    n = x.shape[1]
    w = np.array([0.4, -1.1, 0.7])
    xc = np.array([0.5, 0.4, 0.5])
    v = np.cross(w[None, :], (x - xc[:, None]).T).T
    Sk = np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])
    C = np.tile(Sk.reshape(9, 1), (1, n))
    F = np.tile(np.eye(3).reshape(9, 1), (1, n))
    params = dict(n_grid=32, dt=1e-4, gravity=(0.0, 0.0, 0.0), bc_band=3, material=0,
                  E=1e4, nu=0.3, p_mass=1e-3, p_vol=1e-6)
    wind = (np.zeros((1, 2, 2, 2, 3)), 2, 1, 1.0)
    s = oracle.mpm_substep(params, (x, v, C, F), wind, 0.0)
    assert np.allclose(s[1], v, atol=1e-13)
    assert np.allclose(s[2], C, atol=1e-11)
    assert np.allclose(s[0], x + 1e-4 * v, atol=1e-15)


def test_sticky_walls_stop_particles_in_the_band():
    """A particle whose whole stencil lies in the sticky band gets v = 0."""
    N = 16
    x = np.array([[1.6 / N], [0.5], [0.5]])  # base node 1 in x: nodes 1..3, band 4
    n = 1
    state = (x, np.array([[-1.0], [0.0], [0.0]]), np.zeros((9, n)), np.eye(3).reshape(9, 1).copy())
    params = dict(n_grid=N, dt=1e-3, gravity=(0.0, -9.8, 0.0), bc_band=4, material=0,
                  E=1e3, nu=0.3, p_mass=1e-3, p_vol=1e-6)
    wind = (np.ones((1, 2, 2, 2, 3)), 2, 1, 1.0)
    s = oracle.mpm_substep(params, state, wind, 0.0)
    assert np.abs(s[1]).max() == 0.0
    assert np.array_equal(s[0], x)


def test_pinned_particles_do_not_move():
    params, state = small_scene(n=40, material=0)
    pinned = np.zeros(40, np.uint8)
    pinned[::3] = 1
    wind = (inputs.fourier_wind(4, 2, seed=1).astype(np.float64), 4, 2, 1.0)
    s = oracle.mpm_substep(params, state, wind, 0.3, pinned)
    pm = pinned.astype(bool)
    assert np.array_equal(s[0][:, pm], state[0][:, pm])
    assert np.array_equal(s[3][:, pm], state[3][:, pm])
    assert np.abs(s[1][:, pm]).max() == 0.0 and np.abs(s[2][:, pm]).max() == 0.0
    assert np.abs(s[0][:, ~pm] - state[0][:, ~pm]).max() > 0


def test_out_of_domain_particle_is_an_error():
    params, state = small_scene(n=4)
    x = state[0].copy()
    x[0, 2] = 0.02  # base index -1 on a 12^3 grid
    with pytest.raises(oracle.OracleError):
        oracle.mpm_substep(params, (x,) + state[1:], (np.zeros((1, 2, 2, 2, 3)), 2, 1, 1.0), 0.0)


# ---------------------------------------------------------------- adjoint --

def _fd_check(material, which, n_checks=6, seed=0):
    params, state = small_scene(n=30, N=12, material=material, seed=seed)
    rng = np.random.default_rng(seed + 100)
    nf, nt, T = 4, 3, 0.01
    wv = inputs.fourier_wind(nf, nt, seed=seed).astype(np.float64)
    pinned = (rng.random(30) < 0.2).astype(np.uint8)
    t = 0.004
    g_out = tuple(rng.standard_normal(a.shape) for a in state)

    def loss(st, wvals, E):
        p = dict(params, E=E)
        out = oracle.mpm_substep(p, st, (wvals, nf, nt, T), t, pinned)
        return sum(np.sum(g * o) for g, o in zip(g_out, out))

    g_in, g_w, g_E = oracle.mpm_substep_adjoint(params, state, (wv, nf, nt, T), t, g_out, pinned)
    for _ in range(n_checks):
        if which == "wind":
            k = rng.integers(wv.size)
            h = 1e-4
            wp, wm = wv.copy().ravel(), wv.copy().ravel()
            wp[k] += h
            wm[k] -= h
            fd = (loss(state, wp.reshape(wv.shape), params["E"]) - loss(state, wm.reshape(wv.shape), params["E"])) / (2 * h)
            ad = g_w.ravel()[k]
        elif which == "E":
            h = params["E"] * 1e-6
            fd = (loss(state, wv, params["E"] + h) - loss(state, wv, params["E"] - h)) / (2 * h)
            ad = g_E
        else:
            comp = {"x": 0, "v": 1, "C": 2, "F": 3}[which]
            a = state[comp]
            k = rng.integers(a.size)
            h = 1e-7 if which == "x" else 1e-6
            ap, am = a.copy().ravel(), a.copy().ravel()
            ap[k] += h
            am[k] -= h
            sp = list(state)
            sp[comp] = ap.reshape(a.shape)
            sm = list(state)
            sm[comp] = am.reshape(a.shape)
            fd = (loss(tuple(sp), wv, params["E"]) - loss(tuple(sm), wv, params["E"])) / (2 * h)
            ad = g_in[comp].ravel()[k]
        scale = max(abs(fd), 1e-3 * np.abs(g_in[0]).max() if which == "x" else abs(fd), 1e-12)
        assert abs(ad - fd) <= 1e-5 * scale + 1e-9, (which, ad, fd)


@pytest.mark.parametrize("material", [0, 1])
@pytest.mark.parametrize("which", ["x", "v", "C", "F", "wind", "E"])
def test_substep_adjoint_matches_finite_differences(material, which):
    _fd_check(material, which)
