"""GPU parity of the HOME-LBM step (App. D) against the FP64 oracle
(oracle/home_oracle.c), through the C-ABI. Both sides start from the same
float32 moments; the tolerance is the LBM velocity target (relative L2 over
fluid cells 1e-5), with rho - 1 and S checked against their own scale."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_09668_gb300 import binding as B
from paper_2603_09668_gb300 import inputs

from gpu_util import rel_l2, to_dev

pytestmark = pytest.mark.gpu


def start_moments(shape, tau, u0, force, seed):
    """Collided equilibrium of u0 plus seeded noise on every moment, as the
    float32 device layout (plane 0 = rho - 1) and its float64 oracle copy."""
    rng = np.random.default_rng(seed)
    nc = shape[0] * shape[1] * shape[2]
    m = oracle.home_init(shape, 1.0, u0, tau, force)
    m[0] += 2e-3 * rng.standard_normal(nc)
    m[1:4] += 1e-2 * rng.standard_normal((3, nc))
    m[4:] += 1e-4 * rng.standard_normal((6, nc))
    dev = m.copy()
    dev[0] -= 1.0
    dev = dev.astype(np.float32)
    ref = dev.astype(np.float64)
    ref[0] += 1.0
    return dev, ref


def compare(lbm, m_dev, ref, shape, solid_np, force):
    nx, ny, nz = shape
    solid = None if solid_np is None else to_dev(solid_np).reshape(nz, ny, nx)
    rho, u = lbm.home_macroscopic(m_dev, solid)
    rho_r, u_r = oracle.home_macroscopic(shape, ref, force, solid_np)
    fluid = np.ones(nx * ny * nz, bool) if solid_np is None else solid_np == 0
    u = u.reshape(3, -1).cpu().numpy()[:, fluid]
    assert rel_l2(u, u_r[:, fluid]) <= 1e-5, rel_l2(u, u_r[:, fluid])
    r = rho.reshape(-1).cpu().numpy()[fluid]
    assert np.abs(r - rho_r[fluid]).max() <= 2e-6
    md = m_dev.reshape(10, -1).cpu().numpy().astype(np.float64)[:, fluid]
    S, S_r = md[4:], ref[4:, fluid]
    assert rel_l2(S, S_r) <= 1e-4, rel_l2(S, S_r)


@pytest.mark.parametrize("steps", [1, 8, 9])
def test_home_step_matches_oracle_inlet_mask_force(steps):
    shape = (16, 12, 10)  # no side a multiple of the launch's row
    tau, u_in, force = 0.6, (0.05, 0.02, 0.0), (1e-5, -2e-5, 0.0)
    solid_np = inputs.random_mask(shape, 0.1, seed=21)
    m0, ref0 = start_moments(shape, tau, (0.04, 0.01, 0.0), force, seed=22)
    lbm = B.LBM(shape, tau, u_inlet=u_in, force=force, bc_x=1)
    m = to_dev(m0).reshape(10, shape[2], shape[1], shape[0])
    solid = to_dev(solid_np).reshape(shape[2], shape[1], shape[0])
    lbm.home_step(m, solid, steps)
    ref = oracle.home_step(shape, tau, ref0, steps, u_in=u_in, force=force, bc_x=1,
                           solid=solid_np)
    compare(lbm, m, ref, shape, solid_np, force)
    # solid cells keep their moments bit for bit
    keep = solid_np == 1
    assert np.array_equal(m.reshape(10, -1).cpu().numpy()[:, keep], m0[:, keep])
    lbm.close()


def test_home_step_matches_oracle_periodic():
    shape = (20, 9, 7)
    tau, force = 0.8, (0.0, 0.0, 3e-5)
    m0, ref0 = start_moments(shape, tau, (0.0, 0.03, -0.02), force, seed=23)
    lbm = B.LBM(shape, tau, force=force, bc_x=0)
    m = to_dev(m0).reshape(10, shape[2], shape[1], shape[0])
    lbm.home_step(m, None, 12)
    ref = oracle.home_step(shape, tau, ref0, 12, force=force, bc_x=0)
    compare(lbm, m, ref, shape, None, force)
    lbm.close()


def test_home_step_full_size_leaf_cluster():
    """128^3 with the voxelized leaf cluster and the inlet, two steps."""
    shape = (128, 128, 128)
    tau, u_in = 0.55, (0.05, 0.0, 0.0)
    solid_np = oracle.voxelize(inputs.ellipsoid_cluster(), shape, 1.0 / 128)
    lbm = B.LBM(shape, tau, u_inlet=u_in, bc_x=1)
    m = lbm.moments()
    lbm.home_init(m, 1.0, u_in)
    ref = oracle.home_init(shape, 1.0, u_in, tau)
    ref[0] = 1.0 + m[0].reshape(-1).cpu().numpy().astype(np.float64)  # the float32 start
    ref[1:] = m[1:].reshape(9, -1).cpu().numpy().astype(np.float64)
    solid = to_dev(solid_np).reshape(128, 128, 128)
    lbm.home_step(m, solid, 2)
    ref = oracle.home_step(shape, tau, ref, 2, u_in=u_in, bc_x=1, solid=solid_np)
    compare(lbm, m, ref, shape, solid_np, (0.0, 0.0, 0.0))
    lbm.close()


def test_home_sample_velocity_matches_oracle():
    from oracle import phys

    shape = (16, 12, 10)
    tau, u_in = 0.6, (0.05, 0.02, 0.0)
    solid_np = inputs.random_mask(shape, 0.1, seed=24)
    m0, ref0 = start_moments(shape, tau, (0.04, 0.01, 0.0), (0.0, 0.0, 0.0), seed=25)
    lbm = B.LBM(shape, tau, u_inlet=u_in, bc_x=1)
    m = to_dev(m0).reshape(10, shape[2], shape[1], shape[0])
    solid = to_dev(solid_np).reshape(shape[2], shape[1], shape[0])
    lbm.home_step(m, solid, 5)
    ref = oracle.home_step(shape, tau, ref0, 5, u_in=u_in, bc_x=1, solid=solid_np)
    rng = np.random.default_rng(26)
    pos = np.concatenate([rng.uniform(-0.05, 1.05, (3, 300)), inputs.wind_node_positions(8)],
                         axis=1).astype(np.float32)
    u = lbm.home_sample_velocity(m, solid, to_dev(pos)).cpu().numpy()
    _, u_cells = oracle.home_macroscopic(shape, ref, solid=solid_np)
    u_ref = phys.sample_velocity_field(shape, u_cells, pos.astype(np.float64))
    assert rel_l2(u, u_ref) <= 1e-5, rel_l2(u, u_ref)
    lbm.close()


def test_home_init_matches_oracle_and_argument_errors():
    shape = (6, 5, 4)
    tau, force = 0.7, (2e-5, 0.0, -1e-5)
    lbm = B.LBM(shape, tau, force=force)
    m = lbm.moments()
    lbm.home_init(m, 1.02, (0.03, -0.01, 0.02))
    ref = oracle.home_init(shape, 1.02, (0.03, -0.01, 0.02), tau, force)
    ref[0] -= 1.0
    assert np.allclose(m.reshape(10, -1).cpu().numpy(), ref, rtol=1e-6, atol=1e-9)
    before = m.clone()
    lbm.home_step(m, None, 0)  # no step: unchanged
    assert torch.equal(m, before)
    with pytest.raises(B.DiffWindError):
        lbm.home_step(m, None, -1)
    lbm.close()
