"""GPU parity of the D3Q19 LBM step (AA pattern), its adjoint, the macroscopic
fields and the voxelizer against the FP64 oracle, through the C-ABI.

Tolerances: velocities relative L2 over fluid cells <= 1e-5 (float32 with
shifted populations, f - w, vs float64); adjoint relative L2 <= 1e-4; the
voxel mask is integer work and must match bit for bit."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_09668_gb300 import binding as B
from paper_2603_09668_gb300 import inputs

from gpu_util import rel_l2, to_dev

pytestmark = pytest.mark.gpu


def to_plain(f_shift, w):
    return f_shift.reshape(19, -1).cpu().numpy().astype(np.float64) + w[:, None]


def to_shift(f_plain, w, shape):
    nx, ny, nz = shape
    return to_dev((f_plain - w[:, None]).astype(np.float32).reshape(19, nz, ny, nx))


def fluid_u_error(lbm, f, solid_np, shape, f_ref, force=(0, 0, 0)):
    solid = None if solid_np is None else to_dev(solid_np).reshape(shape[2], shape[1], shape[0])
    _, u = lbm.macroscopic(f, solid)
    _, u_ref = oracle.lbm_macroscopic(shape, f_ref, force=force, solid=solid_np)
    return rel_l2(u.reshape(3, -1).cpu().numpy(), u_ref)


@pytest.mark.parametrize("with_obstacle", [False, True])
def test_inlet_lattice_100_steps(with_obstacle):
    """The forward LBM configuration: 32^3, tau = 0.6, inlet 0.05 in +x,
    periodic y and z, rest start, 100 steps; optionally with the block scene
    voxelized as an obstacle."""
    shape = (32, 32, 32)
    c, w, _ = oracle.velocity_set()
    solid_np = None
    if with_obstacle:
        sc = inputs.block_scene()
        solid_np = oracle.voxelize(sc.x, shape, 1.0 / 32)
    lbm = B.LBM(shape, 0.6, u_inlet=(0.05, 0.0, 0.0), bc_x=1)
    f = lbm.lattice()
    solid = None if solid_np is None else to_dev(solid_np).reshape(32, 32, 32)
    lbm.step(f, solid, 100)
    f_ref = oracle.lbm_step(shape, 0.6, np.repeat(w[:, None], 32 ** 3, axis=1), 100,
                            u_in=(0.05, 0, 0), bc_x=1, solid=solid_np)
    assert fluid_u_error(lbm, f, solid_np, shape, f_ref) <= 1e-5


@pytest.mark.parametrize("steps", [1, 2, 5, 8])
def test_periodic_forced_lattice_with_mask(steps):
    shape = (24, 16, 12)  # ragged against 256-thread blocks
    c, w, _ = oracle.velocity_set()
    solid_np = inputs.random_mask(shape, 0.1, seed=3)
    noise = inputs.population_noise(shape, 2e-3, seed=4).astype(np.float64)
    f0 = w[:, None] + noise
    force = (2e-5, -1e-5, 5e-6)
    lbm = B.LBM(shape, 0.57, force=force, bc_x=0)
    f = to_shift(f0, w, shape)
    lbm.step(f, to_dev(solid_np).reshape(12, 16, 24), steps)
    f_ref = oracle.lbm_step(shape, 0.57, f0, steps, force=force, bc_x=0, solid=solid_np)
    fl = solid_np == 0
    got = to_plain(f, w)
    assert np.abs(got[:, fl] - f_ref[:, fl]).max() <= 2e-7
    assert fluid_u_error(lbm, f, solid_np, shape, f_ref, force) <= 1e-5


def test_inlet_outlet_noise_with_mask_odd_steps():
    shape = (20, 12, 10)
    c, w, _ = oracle.velocity_set()
    solid_np = inputs.random_mask(shape, 0.08, seed=7)
    f0 = w[:, None] + inputs.population_noise(shape, 1e-3, seed=8).astype(np.float64)
    lbm = B.LBM(shape, 0.6, u_inlet=(0.04, 0.01, -0.01), bc_x=1)
    f = to_shift(f0, w, shape)
    lbm.step(f, to_dev(solid_np).reshape(10, 12, 20), 7)
    f_ref = oracle.lbm_step(shape, 0.6, f0, 7, u_in=(0.04, 0.01, -0.01), bc_x=1, solid=solid_np)
    fl = solid_np == 0
    assert np.abs(to_plain(f, w)[:, fl] - f_ref[:, fl]).max() <= 2e-7


def test_full_size_lattice_with_leaf_cluster_four_steps():
    """128^3 lattice, tau = 0.55, inlet 0.05, obstacle from the 200k-particle
    leaf cluster (50 ellipsoids): four steps compared on every cell."""
    shape = (128, 128, 128)
    pts = inputs.ellipsoid_cluster()
    solid_np = oracle.voxelize(pts, shape, 1.0 / 128)
    c, w, _ = oracle.velocity_set()
    lbm = B.LBM(shape, 0.55, u_inlet=(0.05, 0.0, 0.0), bc_x=1)
    f = lbm.lattice()
    u0 = (0.05, 0.0, 0.0)
    lbm.init_equilibrium(f, 1.0, u0)
    solid = to_dev(solid_np).reshape(128, 128, 128)
    lbm.step(f, solid, 4)
    feq = oracle.lbm_equilibrium(1.0, u0)
    f_ref = oracle.lbm_step(shape, 0.55, np.repeat(feq[:, None], 128 ** 3, axis=1), 4,
                            u_in=u0, bc_x=1, solid=solid_np)
    assert fluid_u_error(lbm, f, solid_np, shape, f_ref) <= 1e-5


def test_uniform_flow_stays_uniform_and_mass_is_conserved():
    shape = (64, 32, 16)
    lbm = B.LBM(shape, 0.55, u_inlet=(0.05, 0.0, 0.0), bc_x=1)
    f = lbm.lattice()
    lbm.init_equilibrium(f, 1.0, (0.05, 0.0, 0.0))
    f0 = f.clone()
    lbm.step(f, None, 40)
    assert (f - f0).abs().max().item() <= 1e-7  # float32 rounding of f_eq only
    # closed periodic box with bounce-back obstacles: total mass is conserved
    solid_np = inputs.random_mask(shape, 0.1, seed=1)
    solid = to_dev(solid_np).reshape(16, 32, 64)
    box = B.LBM(shape, 0.6, bc_x=0)
    g = to_dev(inputs.population_noise(shape, 1e-3, seed=2).reshape(19, 16, 32, 64))
    fl = torch.from_numpy(solid_np == 0).cuda().reshape(16, 32, 64)
    m0 = g[:, fl].double().sum().item()
    box.step(g, solid, 30)
    m1 = g[:, fl].double().sum().item()
    assert abs(m1 - m0) <= 1e-7 * fl.sum().item()


@pytest.mark.parametrize("bc_x", [0, 1])
@pytest.mark.parametrize("steps", [1, 4])
def test_step_adjoint_matches_oracle(bc_x, steps):
    shape = (12, 10, 8)
    c, w, _ = oracle.velocity_set()
    solid_np = inputs.random_mask(shape, 0.12, seed=5)
    f0 = w[:, None] + inputs.population_noise(shape, 2e-3, seed=6).astype(np.float64)
    force = (1e-5, 0.0, -2e-5)
    u_in = (0.05, 0.01, 0.0)
    g_end = np.random.default_rng(1).standard_normal((19, np.prod(shape)))
    lbm = B.LBM(shape, 0.6, u_inlet=u_in, force=force, bc_x=bc_x, max_tape=4)
    g = to_dev(g_end.astype(np.float32).reshape(19, 8, 10, 12))
    lbm.step_adjoint(to_shift(f0, w, shape), g, to_dev(solid_np).reshape(8, 10, 12), steps)
    ref = oracle.lbm_step_adjoint(shape, 0.6, f0, g_end, steps, u_in=u_in, force=force, bc_x=bc_x,
                                  solid=solid_np)
    assert rel_l2(g.reshape(19, -1).cpu().numpy().astype(np.float64), ref) <= 1e-4


def test_adjoint_tape_limit_is_an_argument_error():
    lbm = B.LBM((8, 8, 8), 0.6, max_tape=2)
    f = lbm.lattice()
    with pytest.raises(B.DiffWindError, match="DW_ERR_ARG"):
        lbm.step_adjoint(f, f.clone(), None, 3)


def test_voxelize_bit_exact():
    pts = inputs.ellipsoid_cluster(n_patches=10, per_patch=2000, seed=3)
    pts[:, :3] = np.array([[3 / 64, 0.5, 63 / 64], [0.5, 1.0, 0.25], [0.0, -0.01, 0.5]], np.float32).T
    for shape, dx in [((64, 64, 64), 1 / 64), ((40, 24, 16), 1 / 32)]:
        mask = torch.empty(shape[::-1], dtype=torch.uint8, device="cuda")
        B.voxelize_particles(to_dev(pts), shape, dx, mask)
        ref = oracle.voxelize(pts, shape, dx)
        assert np.array_equal(mask.cpu().numpy().ravel(), ref)


def test_cached_mask_link_words():
    """lbm_cache_mask: steps, adjoint and HOME steps with the registered mask
    equal those that rebuild the link words per call, bit for bit; after the
    mask changes and is registered again the steps follow the new mask (a
    stale cache would not)."""
    shape = (24, 16, 12)
    nx, ny, nz = shape
    solid_a = to_dev(inputs.random_mask(shape, 0.1, seed=5)).reshape(nz, ny, nx)
    solid_b = to_dev(inputs.random_mask(shape, 0.1, seed=6)).reshape(nz, ny, nx)
    lbm = B.LBM(shape, 0.6, u_inlet=(0.05, 0.01, 0.0), bc_x=1, max_tape=4)
    f0 = lbm.lattice()
    lbm.init_equilibrium(f0, 1.0, (0.03, 0.0, 0.01))
    ref = f0.clone()
    lbm.step(ref, solid_a, 5)
    g_ref = torch.linspace(-1, 1, f0.numel(), device=f0.device).reshape(f0.shape)
    lbm.step_adjoint(f0, g_ref, solid_a, 4)
    lbm.cache_mask(solid_a)
    f = f0.clone()
    lbm.step(f, solid_a, 5)
    assert torch.equal(f, ref)
    g = torch.linspace(-1, 1, f0.numel(), device=f0.device).reshape(f0.shape)
    lbm.step_adjoint(f0, g, solid_a, 4)
    assert torch.equal(g, g_ref)
    # the mask changes in place: registering it again rebuilds the words
    ref_b = f0.clone()
    lbm.cache_mask(None)
    lbm.step(ref_b, solid_b, 3)
    solid_a.copy_(solid_b)
    lbm.cache_mask(solid_a)
    f = f0.clone()
    lbm.step(f, solid_a, 3)
    assert torch.equal(f, ref_b)
    # HOME steps with the registered mask equal those without
    m0 = lbm.moments()
    lbm.home_init(m0, 1.0, (0.03, 0.0, 0.01))
    m = m0.clone()
    lbm.home_step(m, solid_a, 4)
    lbm.cache_mask(None)
    m_ref = m0.clone()
    lbm.home_step(m_ref, solid_b, 4)
    assert torch.equal(m, m_ref)
    lbm.close()
