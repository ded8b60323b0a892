"""Pins of the HOME-LBM oracle (oracle/home_oracle.c; Sec. 3.4, App. D)
against what the mathematics and the independently pinned BGK oracle fix:

- the reconstruction equals the general Hermite series written as full
  tensor contractions (numpy), and reproduces its moments rho, rho u,
  rho (cs2 I + S) exactly;
- the collision equals the BGK + Guo collision of the same populations
  (oracle.lbm_collide) in rho, momentum and the deviatoric second moment, and
  sets the trace to equilibrium plus half the forcing;
- steps: a uniform flow stays uniform (periodic and inlet/outlet), mass is
  conserved with bounce-back obstacles, a uniform force adds F per cell and
  step, a shear wave decays at the viscosity cs2 (tau - 1/2), and a smooth
  flow converges to the BGK oracle at second order."""
import itertools

import numpy as np
import pytest

import oracle

C, W, _ = oracle.velocity_set()
CS2 = 1.0 / 3.0


def random_moments(rng, n=None, u_scale=0.05, s_scale=2e-3):
    rho = 1.0 + 0.01 * rng.standard_normal()
    u = u_scale * rng.standard_normal(3)
    N = s_scale * rng.standard_normal((3, 3))
    S = np.outer(u, u) + 0.5 * (N + N.T)
    return np.array([rho, *u, S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]])


def s_of(m):
    return np.array([[m[4], m[7], m[8]], [m[7], m[5], m[9]], [m[8], m[9], m[6]]])


def hermite_series(m):
    """w rho [1 + c.u/cs2 + H2:S/(2 cs2^2) + H3:A/(6 cs2^3)] with full tensors."""
    rho, u, S = m[0], m[1:4], s_of(m)
    A = (np.einsum("a,bc->abc", u, S) + np.einsum("b,ac->abc", u, S) +
         np.einsum("c,ab->abc", u, S) - 2 * np.einsum("a,b,c->abc", u, u, u))
    I = np.eye(3)
    f = np.zeros(19)
    for i in range(19):
        c = C[i].astype(np.float64)
        H2 = np.outer(c, c) - CS2 * I
        H3 = (np.einsum("a,b,c->abc", c, c, c) - CS2 * (np.einsum("a,bc->abc", c, I) +
                                                        np.einsum("b,ac->abc", c, I) +
                                                        np.einsum("c,ab->abc", c, I)))
        f[i] = W[i] * rho * (1 + c @ u / CS2 + np.sum(H2 * S) / (2 * CS2 ** 2) +
                             np.sum(H3 * A) / (6 * CS2 ** 3))
    return f


def test_reconstruction_is_the_hermite_series():
    rng = np.random.default_rng(0)
    for _ in range(20):
        m = random_moments(rng)
        assert np.allclose(oracle.home_reconstruct(m), hermite_series(m), rtol=0, atol=1e-15)


def test_reconstruction_moments():
    rng = np.random.default_rng(1)
    for _ in range(20):
        m = random_moments(rng)
        f = oracle.home_reconstruct(m)
        rho, u, S = m[0], m[1:4], s_of(m)
        assert f.sum() == pytest.approx(rho, abs=1e-14)
        assert np.allclose(C.T @ f, rho * u, atol=1e-15)
        Pi = np.einsum("ia,ib,i->ab", C, C, f)
        assert np.allclose(Pi, rho * (CS2 * np.eye(3) + S), atol=1e-15)


def test_reconstruction_is_cubic_symmetric():
    rng = np.random.default_rng(2)
    m = random_moments(rng)
    f = oracle.home_reconstruct(m)
    key = {tuple(c): i for i, c in enumerate(C)}
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            Q = np.zeros((3, 3))
            for a in range(3):
                Q[a, perm[a]] = signs[a]
            u2 = Q @ m[1:4]
            S2 = Q @ s_of(m) @ Q.T
            m2 = np.array([m[0], *u2, S2[0, 0], S2[1, 1], S2[2, 2], S2[0, 1], S2[0, 2], S2[1, 2]])
            f2 = oracle.home_reconstruct(m2)
            for i in range(19):
                j = key[tuple((Q @ C[i]).astype(int))]
                assert f2[j] == pytest.approx(f[i], abs=1e-15)


@pytest.mark.parametrize("tau", [0.55, 0.8, 1.0, 1.7])
def test_collision_matches_bgk_except_the_trace(tau):
    rng = np.random.default_rng(3)
    force = np.array([2e-4, -1e-4, 3e-4])
    for _ in range(5):
        f = oracle.lbm_equilibrium(1.0 + 0.01 * rng.standard_normal(), 0.05 * rng.standard_normal(3))
        f = f + 1e-3 * rng.standard_normal(19) * W  # non-equilibrium parts of every order
        m = oracle.home_collide(f, tau, force)
        fb = oracle.lbm_collide(f, tau, force)
        rho = m[0]
        assert rho == pytest.approx(fb.sum(), abs=1e-14)
        # stored velocity u' = (momentum after the BGK collision) / rho
        assert np.allclose(rho * m[1:4], C.T @ fb, atol=1e-15)
        Pi = rho * (CS2 * np.eye(3) + s_of(m))
        Pb = np.einsum("ia,ib,i->ab", C, C, fb)
        dev = lambda X: X - np.trace(X) / 3 * np.eye(3)
        assert np.allclose(dev(Pi), dev(Pb), atol=1e-15)
        # trace: equilibrium plus half the forcing moment
        u = (C.T @ f + 0.5 * force) / f.sum()
        tr_eq = 3 * rho * CS2 + rho * u @ u
        assert np.trace(Pi) == pytest.approx(tr_eq + u @ force, abs=1e-15)


def test_collision_relaxes_the_deviatoric_part_at_one_over_tau():
    rng = np.random.default_rng(4)
    tau = 0.7
    m0 = random_moments(rng)
    f = oracle.home_reconstruct(m0)  # populations with non-equilibrium S
    m = oracle.home_collide(f, tau)
    u = m0[1:4]
    Neq = s_of(m0) - np.outer(u, u)
    dev = Neq - np.trace(Neq) / 3 * np.eye(3)
    assert np.allclose(m[1:4], u, atol=1e-16)
    assert np.allclose(s_of(m), np.outer(u, u) + (1 - 1 / tau) * dev, atol=1e-16)


def test_uniform_flow_stays_uniform():
    shape = (6, 5, 4)
    nc = 120
    for bc_x, u0 in ((0, (0.04, -0.01, 0.02)), (1, (0.05, 0.0, 0.01))):
        m = oracle.home_init(shape, 1.0, u0, 0.6)
        m2 = oracle.home_step(shape, 0.6, m, 10, u_in=u0, bc_x=bc_x)
        assert np.allclose(m2, m, atol=1e-14)
        rho, u = oracle.home_macroscopic(shape, m2)
        assert np.allclose(u, np.asarray(u0)[:, None], atol=1e-14)
        assert rho.shape == (nc,)


def test_mass_is_conserved_with_obstacles():
    shape = (8, 7, 6)
    nc = 8 * 7 * 6
    rng = np.random.default_rng(5)
    solid = (rng.random(nc) < 0.15).astype(np.uint8)
    m = oracle.home_init(shape, 1.0, (0.03, 0.01, -0.02), 0.65)
    m[0] += 0.01 * rng.standard_normal(nc)
    m2 = oracle.home_step(shape, 0.65, m, 15, solid=solid)
    fluid = solid == 0
    assert m2[0, fluid].sum() == pytest.approx(m[0, fluid].sum(), abs=1e-11)
    assert np.array_equal(m2[:, ~fluid], m[:, ~fluid])  # solid cells untouched


def test_uniform_force_adds_momentum():
    shape = (4, 4, 4)
    force = np.array([1e-4, -2e-4, 5e-5])
    m = oracle.home_init(shape, 1.0, (0.01, 0.0, 0.0), 0.8, force)
    rho0, u0 = oracle.home_macroscopic(shape, m, force)
    m2 = oracle.home_step(shape, 0.8, m, 7, force=force)
    rho, u = oracle.home_macroscopic(shape, m2, force)
    assert np.allclose(rho * u, rho0 * u0 + 7 * force[:, None], atol=1e-15)


def shear_wave_amplitude(shape, tau, steps, amp=1e-3):
    nx, ny, nz = shape
    y = (np.arange(ny) + 0.0)
    ux = amp * np.sin(2 * np.pi * y / ny)
    m = oracle.home_init(shape, 1.0, (0.0, 0.0, 0.0), tau)
    ux_cells = np.tile(np.repeat(ux, nx), nz)
    m[1] = ux_cells
    m[4] = ux_cells ** 2
    m = oracle.home_step(shape, tau, m, steps)
    _, u = oracle.home_macroscopic(shape, m)
    prof = u[0].reshape(nz, ny, nx)[0, :, 0]
    return 2 * np.mean(prof * np.sin(2 * np.pi * y / ny)), m


@pytest.mark.parametrize("tau", [0.6, 0.9])
def test_shear_wave_decays_at_the_bgk_viscosity(tau):
    shape, steps = (2, 32, 1), 300
    a, _ = shear_wave_amplitude(shape, tau, steps)
    nu = CS2 * (tau - 0.5)
    k = 2 * np.pi / 32
    expect = 1e-3 * np.exp(-nu * k * k * steps)
    assert a == pytest.approx(expect, rel=5e-3)


def home_bgk_gap(shape, steps, tau=0.7, amp=0.01):
    """Relative L2 gap of the velocity after `steps` between the HOME and the
    BGK oracle, both started from the equilibrium of a smooth periodic field
    (BGK takes it as pre-collision populations, HOME stores it collided)."""
    nx, ny, nz = shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    u = amp * np.stack([2 * np.sin(2 * np.pi * yy / ny), 1.5 * np.cos(2 * np.pi * zz / nz),
                        np.sin(2 * np.pi * xx / nx)]).reshape(3, -1)
    f = np.stack([oracle.lbm_equilibrium(1.0, u[:, c]) for c in range(u.shape[1])], axis=1)
    m = np.stack([oracle.home_collide(f[:, c], tau) for c in range(f.shape[1])], axis=1)
    _, ub = oracle.lbm_macroscopic(shape, oracle.lbm_step(shape, tau, f, steps))
    _, uh = oracle.home_macroscopic(shape, oracle.home_step(shape, tau, m, steps))
    return np.linalg.norm(uh - ub) / np.linalg.norm(ub)


def test_smooth_flow_converges_to_the_bgk_oracle():
    """Both solve the same Navier-Stokes limit with the same shear viscosity:
    the gap shrinks at second order (doubling the grid, four times the steps
    for the same viscous time, divides it by about four)."""
    coarse = home_bgk_gap((12, 10, 8), 40)
    fine = home_bgk_gap((24, 20, 16), 160)
    assert fine < 6e-3 and fine < 0.3 * coarse, (coarse, fine)
