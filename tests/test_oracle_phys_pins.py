"""Pins of the physics-informed wind loss oracle (oracle/phys.py) against
what Sec. 3.4 and the mathematics fix: closed forms of L_phys (a force along
the flow costs nothing, a force across it costs |F|^2), its invariance under
rotations, its gradient by central differences; the guide velocity sampler
against lattices whose velocity field is known in closed form (uniform and
linear fields are reproduced exactly by trilinear interpolation, solid cells
are at rest); the drag relation by its closed form along an axis, its degree-2
homogeneity and its direction; the trajectory term's gradient by central
differences; Adam against torch.optim.Adam (an independent implementation);
VectorAdam against torch's Adam where each vector's gradient stays on one
axis (the two then agree) and by its rotation equivariance."""
import numpy as np
import pytest
import torch

import oracle
from oracle import phys


def eq_lattice(shape, ufun):
    """Populations f_eq(1, u(cell centre)) of every cell (the lattice oracle's
    natural order), so that the macroscopic velocity is u exactly."""
    nx, ny, nz = shape
    f = np.zeros((19, nz * ny * nx))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                c = (z * ny + y) * nx + x
                u = ufun((x + 0.5) / nx, (y + 0.5) / ny, (z + 0.5) / nz)
                f[:, c] = oracle.lbm_equilibrium(1.0, u)
    return f


def test_uniform_flow_is_sampled_exactly():
    shape = (6, 5, 4)
    u0 = np.array([0.03, -0.01, 0.02])
    f = eq_lattice(shape, lambda x, y, z: u0)
    pos = np.random.default_rng(0).random((3, 50))
    u = phys.lbm_sample_velocity(shape, f, pos)
    assert np.allclose(u, u0[:, None], atol=1e-15)


def test_linear_field_is_reproduced_between_cell_centres():
    shape = (8, 6, 5)
    a = np.array([[0.02, -0.01, 0.005], [0.0, 0.015, -0.01], [0.01, 0.0, 0.02]])
    b = np.array([0.01, -0.02, 0.005])
    f = eq_lattice(shape, lambda x, y, z: b + a @ np.array([x, y, z]))
    rng = np.random.default_rng(1)
    # points inside the box of cell centres
    lo = np.array([0.5 / shape[0], 0.5 / shape[1], 0.5 / shape[2]])
    pos = lo[:, None] + rng.random((3, 40)) * (1 - 2 * lo)[:, None]
    u = phys.lbm_sample_velocity(shape, f, pos)
    assert np.allclose(u, b[:, None] + a @ pos, atol=1e-14)
    # outside that box the point is clamped to the nearest centre
    out = phys.lbm_sample_velocity(shape, f, np.array([[0.0], [0.0], [0.0]]))
    assert np.allclose(out[:, 0], b + a @ lo, atol=1e-14)


def test_solid_cells_are_at_rest():
    shape = (4, 4, 4)
    u0 = np.array([0.04, 0.0, 0.0])
    f = eq_lattice(shape, lambda x, y, z: u0)
    solid = np.zeros(64, np.uint8)
    solid[(1 * 4 + 1) * 4 + 1] = 1  # cell (1, 1, 1)
    # the centre of cell (1, 1, 1) samples that cell alone
    u = phys.lbm_sample_velocity(shape, f, np.array([[1.5 / 4], [1.5 / 4], [1.5 / 4]]), solid)
    assert np.allclose(u, 0.0)
    # half way to cell (2, 1, 1): the mean of rest and u0
    u = phys.lbm_sample_velocity(shape, f, np.array([[2.0 / 4], [1.5 / 4], [1.5 / 4]]), solid)
    assert np.allclose(u[:, 0], 0.5 * u0)


def test_phys_loss_closed_forms():
    rng = np.random.default_rng(2)
    u = rng.standard_normal((3, 20))
    d = u / np.linalg.norm(u, axis=0)
    along = (3.0 * d).T
    loss, g = phys.phys_loss(along, u)
    assert loss == pytest.approx(0.0, abs=1e-24)
    assert np.allclose(g, 0.0, atol=1e-12)
    # a force across the flow costs all of its square
    perp = np.cross(d.T, rng.standard_normal((20, 3)))
    loss, g = phys.phys_loss(perp, u)
    assert loss == pytest.approx(float(np.sum(perp ** 2)), rel=1e-12)
    assert np.allclose(g, 2 * perp, atol=1e-12)
    # still nodes give no guidance
    loss, g = phys.phys_loss(perp, np.zeros((3, 20)))
    assert loss == 0.0 and not g.any()


def test_phys_loss_is_rotation_invariant():
    rng = np.random.default_rng(3)
    F = rng.standard_normal((30, 3))
    u = rng.standard_normal((3, 30))
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    l0, g0 = phys.phys_loss(F, u)
    l1, g1 = phys.phys_loss(F @ q.T, q @ u)
    assert l1 == pytest.approx(l0, rel=1e-12)
    assert np.allclose(g1, g0 @ q.T, atol=1e-12)


def test_phys_loss_gradient_by_central_differences():
    rng = np.random.default_rng(4)
    F = rng.standard_normal((12, 3))
    u = rng.standard_normal((3, 12))
    u[:, 5] = 0.0  # a still node
    _, g = phys.phys_loss(F, u)
    eps = 1e-6
    for k in range(12):
        for c in range(3):
            Fp, Fm = F.copy(), F.copy()
            Fp[k, c] += eps
            Fm[k, c] -= eps
            fd = (phys.phys_loss(Fp, u)[0] - phys.phys_loss(Fm, u)[0]) / (2 * eps)
            assert g[k, c] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_adam_matches_torch():
    rng = np.random.default_rng(5)
    p0 = rng.standard_normal(17)
    grads = [rng.standard_normal(17) for _ in range(6)]
    p, m, v = p0.copy(), np.zeros(17), np.zeros(17)
    t = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=0.05, betas=(0.9, 0.999), eps=1e-8)
    for k, g in enumerate(grads, start=1):
        p, m, v = phys.adam_step(p, g, m, v, k, 0.05)
        opt.zero_grad()
        t.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
    assert np.allclose(p, t.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_scores():
    a = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    assert phys.cos_sim(a, a) == pytest.approx(1.0)
    assert phys.cos_sim(a, -a) == pytest.approx(-1.0)
    assert phys.cos_sim(a, np.array([[0.0, 1.0, 0.0], [3.0, 0.0, 0.0]])) == pytest.approx(0.0)
    assert phys.nmse(a, a) == 0.0
    assert phys.nmse(5 * a, a) == pytest.approx(0.0)  # directions only
    assert phys.nmse(-a, a) == pytest.approx(4.0)
    # unit vectors: |a^ - b^|^2 = 2 - 2 a^.b^, so NMSE = 2 - 2 CosSim
    rng = np.random.default_rng(6)
    x, y = rng.standard_normal((50, 3)), rng.standard_normal((50, 3))
    assert phys.nmse(x, y) == pytest.approx(2 - 2 * phys.cos_sim(x, y), abs=1e-12)
    # a location without a direction is left out
    z = x.copy()
    z[3] = 0.0
    assert phys.cos_sim(z, y) == pytest.approx(phys.cos_sim(np.delete(x, 3, 0), np.delete(y, 3, 0)))


def test_drag_force_closed_form_and_homogeneity():
    # along +x: F = scale u^2, no other component; the sign follows u
    F = phys.drag_force(np.array([[0.05, -0.05], [0.0, 0.0], [0.0, 0.0]]), 4000.0)
    assert np.allclose(F, [[10.0, 0.0, 0.0], [-10.0, 0.0, 0.0]], atol=1e-12)
    rng = np.random.default_rng(7)
    u = rng.standard_normal((3, 25))
    F = phys.drag_force(u, 2.0)
    # |F| = scale |u|^2, parallel to u, degree 2 in u
    assert np.allclose(np.linalg.norm(F, axis=1), 2.0 * np.sum(u * u, axis=0), rtol=1e-12)
    assert np.allclose(np.cross(F, u.T), 0.0, atol=1e-12)
    assert np.all(np.sum(F * u.T, axis=1) >= 0)
    assert np.allclose(phys.drag_force(3.0 * u, 2.0), 9.0 * F, rtol=1e-12)
    assert not phys.drag_force(np.zeros((3, 4)), 2.0).any()


def test_position_loss_closed_form_and_gradient():
    x = np.array([[0.5, 0.2], [0.1, 0.3], [0.0, 0.4]])
    t = np.array([[0.5, 0.0], [0.4, 0.3], [0.0, 0.0]])
    loss, g = phys.position_loss(x, t, weight=2.0)
    assert loss == pytest.approx(2.0 * (0.09 + 0.04 + 0.16))
    rng = np.random.default_rng(8)
    x, t = rng.random((3, 6)), rng.random((3, 6))
    _, g = phys.position_loss(x, t, weight=0.7)
    eps = 1e-6
    for c in range(3):
        for p in range(6):
            xp, xm = x.copy(), x.copy()
            xp[c, p] += eps
            xm[c, p] -= eps
            fd = (phys.position_loss(xp, t, 0.7)[0] - phys.position_loss(xm, t, 0.7)[0]) / (2 * eps)
            assert g[c, p] == pytest.approx(fd, rel=1e-6)


def test_vector_adam_reduces_to_adam_on_axis_aligned_gradients():
    rng = np.random.default_rng(9)
    n = 10
    axis = rng.integers(0, 3, n)
    p0 = rng.standard_normal((n, 3))
    p, m, v = p0.copy(), np.zeros((n, 3)), np.zeros(n)
    t = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=0.03)
    for k in range(1, 7):
        g = np.zeros((n, 3))
        g[np.arange(n), axis] = rng.standard_normal(n)
        p, m, v = phys.vector_adam_step(p, g, m, v, k, 0.03)
        opt.zero_grad()
        t.grad = torch.tensor(g)
        opt.step()
    # components that never saw a gradient stay put in both
    assert np.allclose(p, t.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_vector_adam_is_rotation_equivariant():
    rng = np.random.default_rng(10)
    n = 8
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    p, m, v = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    pr, mr, vr = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    for k in range(1, 6):
        g = rng.standard_normal((n, 3))
        p, m, v = phys.vector_adam_step(p, g, m, v, k, 0.1)
        pr, mr, vr = phys.vector_adam_step(pr, g @ q.T, mr, vr, k, 0.1)
    assert np.allclose(pr, p @ q.T, atol=1e-12)
    # the first step moves each vector by lr along -g/|g| (up to eps)
    g = rng.standard_normal((n, 3))
    p1, _, _ = phys.vector_adam_step(np.zeros((n, 3)), g, np.zeros((n, 3)), np.zeros(n), 1, 0.1)
    assert np.allclose(p1, -0.1 * g / np.linalg.norm(g, axis=1)[:, None], atol=1e-9)


def test_wind_node_positions_are_the_wind_field_nodes():
    """The guide is sampled at inputs.wind_node_positions; sampling the wind
    field there must return its node values exactly (same node order, x
    fastest), so L_phys compares each node's force with the flow at that node."""
    from paper_2603_09668_gb300 import inputs

    nf = 5
    vals = inputs.fourier_wind(nf, 1, seed=3).astype(np.float64)
    pos = inputs.wind_node_positions(nf).astype(np.float64)
    got = oracle.wind_sample(vals, nf, 1, 1.0, pos, 0.0)
    assert np.allclose(got.T, vals[0].reshape(-1, 3), atol=1e-12)


def test_gaussian_scene_ties_are_exact():
    from paper_2603_09668_gb300 import inputs

    x, *_ = inputs.gaussian_scene(n=40, depth_ties=True, seed=1)
    assert np.array_equal(x[2, 4::4], x[2, 3:-1:4][: len(x[2, 4::4])])
