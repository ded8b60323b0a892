"""Pins for the FP64 LBM oracle and the voxelizer against what the method and
the mathematics fix: lattice symmetries, equilibrium moments, conservation,
Guo forcing's momentum input, exact uniform flow, the closed-form Poiseuille
profile, finite differences for the adjoint and brute force for the mask."""
import numpy as np
import pytest

import oracle
from paper_2603_09668_gb300 import inputs

RNG = np.random.default_rng(77)


def test_velocity_set_symmetries():
    c, w, op = oracle.velocity_set()
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.all(c[op] == -c)
    assert np.allclose((w[:, None] * c).sum(0), 0.0)
    # second moment sum w c c = c_s^2 I with c_s^2 = 1/3
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3.0, atol=1e-15)
    # fourth-moment isotropy of D3Q19: sum w c_a^4 = 1/3, sum w c_a^2 c_b^2 = 1/9
    assert np.einsum("i,i->", w, c[:, 0] ** 4) == pytest.approx(1 / 3)
    assert np.einsum("i,i->", w, c[:, 0] ** 2 * c[:, 1] ** 2) == pytest.approx(1 / 9)
    assert sorted(map(tuple, c)) == sorted(
        [(0, 0, 0)] + [tuple(v) for v in np.vstack([np.eye(3), -np.eye(3)]).astype(int)] +
        [(a, b, 0) for a in (-1, 1) for b in (-1, 1)] + [(a, 0, b) for a in (-1, 1) for b in (-1, 1)] +
        [(0, a, b) for a in (-1, 1) for b in (-1, 1)])


@pytest.mark.parametrize("rho,u", [(1.0, (0.0, 0.0, 0.0)), (1.03, (0.05, -0.02, 0.01)),
                                   (0.97, (-0.1, 0.07, 0.03))])
def test_equilibrium_moments(rho, u):
    c, w, _ = oracle.velocity_set()
    u = np.array(u)
    feq = oracle.lbm_equilibrium(rho, u)
    assert feq.sum() == pytest.approx(rho, abs=1e-15)
    assert np.allclose(c.T @ feq, rho * u, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib->ab", feq, c, c), rho * (np.eye(3) / 3 + np.outer(u, u)),
                       atol=1e-15)


def test_collision_conserves_mass_momentum_and_adds_force():
    c, w, _ = oracle.velocity_set()
    for force in [(0.0, 0.0, 0.0), (1e-4, -3e-5, 2e-5)]:
        f = oracle.lbm_equilibrium(1.0, (0.04, 0.01, -0.02)) + RNG.uniform(-1e-3, 1e-3, 19)
        fp = oracle.lbm_collide(f, 0.6, force)
        assert fp.sum() == pytest.approx(f.sum(), abs=1e-15)
        assert np.allclose(c.T @ fp - c.T @ f, force, atol=1e-15)


def test_collision_relaxes_to_equilibrium_at_tau_one():
    f = oracle.lbm_equilibrium(1.01, (0.03, 0.0, 0.02)) + RNG.uniform(-1e-3, 1e-3, 19)
    c, _, _ = oracle.velocity_set()
    rho = f.sum()
    u = c.T @ f / rho
    assert np.allclose(oracle.lbm_collide(f, 1.0), oracle.lbm_equilibrium(rho, u), atol=1e-16)


def test_uniform_flow_stays_uniform_with_inlet_and_outlet():
    shape = (12, 6, 5)
    u_in = np.array([0.05, 0.0, 0.0])
    feq = oracle.lbm_equilibrium(1.0, u_in)
    f = np.repeat(feq[:, None], np.prod(shape), axis=1)
    out = oracle.lbm_step(shape, 0.6, f, 30, u_in=u_in, bc_x=1)
    assert np.abs(out - f).max() < 1e-15


def test_mass_conservation_periodic_with_bounce_back():
    shape = (10, 8, 6)
    nc = np.prod(shape)
    solid = inputs.random_mask(shape, 0.15, seed=2)
    c, w, _ = oracle.velocity_set()
    f = w[:, None] + inputs.population_noise(shape, 1e-3, seed=3).astype(np.float64)
    out = oracle.lbm_step(shape, 0.7, f, 25, bc_x=0, solid=solid)
    fluid = solid == 0
    assert out[:, fluid].sum() == pytest.approx(f[:, fluid].sum(), rel=1e-14)
    assert np.array_equal(out[:, ~fluid], f[:, ~fluid])  # solid populations untouched


def test_streaming_moves_populations_one_link():
    """With tau = 1 on a lattice at equilibrium except one tagged population,
    streaming alone is observable: start from f = f_eq(1, 0) and check that a
    uniform state is a fixed point, then that a pure streaming displacement of
    a post-collision field lands one node along c_i (periodic)."""
    shape = (5, 4, 3)
    nc = np.prod(shape)
    c, w, _ = oracle.velocity_set()
    f = np.repeat(w[:, None], nc, axis=1)
    assert np.abs(oracle.lbm_step(shape, 1.0, f, 3) - f).max() < 1e-16
    # a single-node density bump: after one step with tau = 1 the post-collision
    # populations are f_eq(rho, u) at that node and travel to x + c_i
    g = f.copy()
    node = (2, 1, 1)
    cell = (node[2] * shape[1] + node[1]) * shape[0] + node[0]
    g[:, cell] *= 1.1
    out = oracle.lbm_step(shape, 1.0, g, 1)
    post = oracle.lbm_collide(g[:, cell], 1.0)
    for i in range(19):
        tx = (node[0] + c[i, 0]) % shape[0]
        ty = (node[1] + c[i, 1]) % shape[1]
        tz = (node[2] + c[i, 2]) % shape[2]
        tcell = (tz * shape[1] + ty) * shape[0] + tx
        assert out[i, tcell] == pytest.approx(post[i], abs=1e-16)


def test_poiseuille_channel_closed_form():
    """Body-force channel between halfway bounce-back walls: u(y) =
    F/(2 nu) (y - y0)(H - (y - y0)), nu = (tau - 1/2)/3. At tau = 1/2 +
    sqrt(3/16) the BGK wall location is exact, so the steady profile matches to
    round-off once converged."""
    ny = 18
    shape = (2, ny, 1)
    H = ny - 2
    tau = 0.5 + np.sqrt(3.0 / 16.0)
    nu = (tau - 0.5) / 3.0
    Fx = 1e-6
    solid = np.zeros(ny * 2, np.uint8).reshape(1, ny, 2)
    solid[:, 0, :] = 1
    solid[:, -1, :] = 1
    c, w, _ = oracle.velocity_set()
    f = np.repeat(w[:, None], 2 * ny, axis=1)
    f = oracle.lbm_step(shape, tau, f, 12000, force=(Fx, 0, 0), bc_x=0, solid=solid.ravel())
    rho, u = oracle.lbm_macroscopic(shape, f, force=(Fx, 0, 0), solid=solid.ravel())
    y = np.arange(ny) - 0.5  # wall halfway between node 0 and node 1
    exact = Fx / (2 * nu) * y * (H - y)
    ux = u[0].reshape(ny, 2)[1:-1, 0]
    assert np.abs(ux - exact[1:-1]).max() < 1e-9 * exact.max()
    # and a generic tau is second-order close (not exact)
    tau2 = 0.8
    nu2 = (tau2 - 0.5) / 3.0
    f2 = oracle.lbm_step(shape, tau2, np.repeat(w[:, None], 2 * ny, axis=1), 6000,
                         force=(Fx, 0, 0), bc_x=0, solid=solid.ravel())
    _, u2 = oracle.lbm_macroscopic(shape, f2, force=(Fx, 0, 0), solid=solid.ravel())
    exact2 = Fx / (2 * nu2) * y * (H - y)
    err = np.abs(u2[0].reshape(ny, 2)[1:-1, 0] - exact2[1:-1]).max() / exact2.max()
    assert 1e-6 < err < 2e-2


def test_collision_adjoint_finite_differences():
    for force in [(0.0, 0.0, 0.0), (2e-4, 1e-4, -1e-4)]:
        f = oracle.lbm_equilibrium(1.02, (0.05, -0.03, 0.02)) + RNG.uniform(-2e-3, 2e-3, 19)
        gpost = RNG.standard_normal(19)
        gpre = oracle.lbm_collide_adjoint(f, 0.57, gpost, force)
        h = 1e-7
        for j in range(19):
            fp, fm = f.copy(), f.copy()
            fp[j] += h
            fm[j] -= h
            fd = (gpost @ oracle.lbm_collide(fp, 0.57, force) - gpost @ oracle.lbm_collide(fm, 0.57, force)) / (2 * h)
            assert gpre[j] == pytest.approx(fd, rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("bc_x", [0, 1])
def test_step_adjoint_finite_differences(bc_x):
    shape = (6, 5, 4)
    nc = np.prod(shape)
    solid = inputs.random_mask(shape, 0.15, seed=4)
    c, w, _ = oracle.velocity_set()
    f0 = w[:, None] + inputs.population_noise(shape, 2e-3, seed=5).astype(np.float64)
    u_in = (0.05, 0.01, 0.0)
    force = (1e-5, 0.0, -2e-5)
    g_end = RNG.standard_normal((19, nc))
    steps = 3
    g0 = oracle.lbm_step_adjoint(shape, 0.6, f0, g_end, steps, u_in=u_in, force=force, bc_x=bc_x, solid=solid)

    def loss(f):
        return np.sum(g_end * oracle.lbm_step(shape, 0.6, f, steps, u_in=u_in, force=force, bc_x=bc_x, solid=solid))

    rng = np.random.default_rng(9)
    for _ in range(12):
        k = rng.integers(f0.size)
        h = 1e-6
        fp, fm = f0.copy().ravel(), f0.copy().ravel()
        fp[k] += h
        fm[k] -= h
        fd = (loss(fp.reshape(f0.shape)) - loss(fm.reshape(f0.shape))) / (2 * h)
        assert g0.ravel()[k] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_voxelize_brute_force_eq_point2voxel():
    shape = (8, 7, 6)
    dx = 1.0 / 8.0  # lattice spacings are 1/N with N a power of two: exact
    pos = RNG.uniform(-0.05, 0.95, (3, 40))
    pos[:, 0] = [3 / 8, 4 / 8, 5 / 8]  # exactly on cell faces: belongs to the higher cell
    mask = oracle.voxelize(pos, shape, dx)
    nx, ny, nz = shape
    expect = np.zeros(nx * ny * nz, np.uint8)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                xw = np.array([x, y, z]) * dx
                d = pos - xw[:, None]
                if np.any(np.all((d >= 0) & (d < dx), axis=0)):
                    expect[(z * ny + y) * nx + x] = 1
    assert np.array_equal(mask, expect)
    assert mask[(5 * ny + 4) * nx + 3] == 1
