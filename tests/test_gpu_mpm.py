"""GPU parity of the MPM substep, its adjoint, the wind sampler and the
particle sort against the FP64 oracle, through the C-ABI.

Tolerances (float32 path vs float64 oracle):
  positions after 100 substeps       max |dx| <= 1e-4 (of the unit domain)
  one substep, per field             max |d| / max |ref|: x 1e-6 (absolute),
                                     v 1e-4, C 2e-3, F 1e-6 (absolute)
  adjoint gradients                  relative L2 <= 1e-4 per gradient block
                                     (x, v, C, F, wind values, E)
The single-substep bounds follow from float32 rounding (2^-24 relative) of
sums of 27 terms whose magnitudes exceed the result by the APIC cancellation
factor 4/dx^2 * dx^2 / 4 ~ 1 for C and by ~1e3 for the stress momentum.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_09668_gb300 import binding as B
from paper_2603_09668_gb300 import inputs

from gpu_util import f64, max_rel, rel_l2, state_to_dev, state_to_np, to_dev, wind_dev, wind_ref

pytestmark = pytest.mark.gpu

MODES = [B.P2G_ATOMIC, B.P2G_WARP, B.P2G_TILE]


def perturbed_block(n_sub=8, material=1, seed=3, N=32):
    x = inputs.block_particles(sub=n_sub, per_sub=2, seed=seed)
    st = inputs.perturbed_state(x, v_scale=0.05, c_scale=0.5, f_scale=0.01, seed=seed)
    params = dict(n_grid=N, dt=1e-4, gravity=(0.0, -9.8, 0.0), bc_band=3, material=material,
                  E=1e4, nu=0.3, p_mass=1000.0 * 0.25 ** 3 / x.shape[1], p_vol=0.25 ** 3 / x.shape[1])
    return params, st


def check_state(gpu, ref, label=""):
    g = state_to_np(gpu)
    assert np.abs(g[0] - ref[0]).max() <= 1e-6, (label, "x", np.abs(g[0] - ref[0]).max())
    assert max_rel(g[1], ref[1]) <= 1e-4, (label, "v", max_rel(g[1], ref[1]))
    assert max_rel(g[2], ref[2]) <= 2e-3, (label, "C", max_rel(g[2], ref[2]))
    assert np.abs(g[3] - ref[3]).max() <= 1e-6, (label, "F", np.abs(g[3] - ref[3]).max())


# ------------------------------------------------------------------- wind --

@pytest.mark.parametrize("nf,nt", [(8, 1), (5, 4), (32, 16), (1, 3)])
def test_wind_sample_matches_oracle(nf, nt):
    vals = inputs.fourier_wind(nf, nt, seed=nf + nt)
    rng = np.random.default_rng(0)
    pos = rng.uniform(-0.2, 1.2, (3, 1000)).astype(np.float32)
    T = 0.05
    w = wind_dev(vals, T)
    for t in [-0.01, 0.0, 0.013, 0.05, 0.07]:
        out = B.wind_field_sample(w, to_dev(pos), t).cpu().numpy()
        ref = oracle.wind_sample(vals, nf, nt, T, pos, t)
        assert np.abs(out - ref).max() <= 2e-6 * np.abs(vals).max()


def test_wind_sample_adjoint_matches_oracle():
    nf, nt, T = 6, 5, 1.0
    vals = inputs.fourier_wind(nf, nt, seed=4)
    rng = np.random.default_rng(1)
    pos = rng.uniform(-0.1, 1.1, (3, 3000)).astype(np.float32)
    g = rng.standard_normal((3, 3000)).astype(np.float32)
    gv = torch.zeros(vals.shape, dtype=torch.float32, device="cuda")
    B.wind_field_sample_adjoint(wind_dev(vals, T), to_dev(pos), 0.37, to_dev(g), gv)
    ref = oracle.wind_sample_adjoint(vals, nf, nt, T, pos, 0.37, g)
    assert rel_l2(gv.cpu().numpy(), ref) <= 1e-5


def test_wind_sample_empty_and_bad_arguments():
    w = wind_dev(inputs.constant_wind(4, 1, (1, 2, 3)), 1.0)
    out = torch.empty((3, 0), device="cuda")
    B.wind_field_sample(w, torch.empty((3, 0), device="cuda"), 0.0, out)
    bad = B.WindField(torch.zeros((2, 4, 4, 4, 3), device="cuda"), 0.0)  # t_total must be > 0
    with pytest.raises(B.DiffWindError):
        B.wind_field_sample(bad, torch.zeros((3, 4), device="cuda"), 0.0)


# ---------------------------------------------------------------- forward --

@pytest.mark.parametrize("material", [0, 1])
@pytest.mark.parametrize("mode", MODES)
def test_one_substep_matches_oracle(material, mode):
    params, st = perturbed_block(material=material)
    vals = inputs.fourier_wind(8, 4, seed=7)
    n = st[0].shape[1]
    pinned = (np.random.default_rng(2).random(n) < 0.1).astype(np.uint8)
    mpm = B.MPM.from_params(params, max_particles=n, p2g_mode=mode)
    out = B.MpmState.empty_like(state_to_dev(st))
    mpm.substep(state_to_dev(st), out, to_dev(pinned), wind_dev(vals, 0.01), 0.0042)
    mpm.device_status()
    ref = oracle.mpm_substep(params, f64(st), wind_ref(vals, 0.01), 0.0042, pinned)
    check_state(out, ref, f"material={material} mode={mode}")


@pytest.mark.parametrize("mode", MODES)
def test_in_place_substep_equals_out_of_place(mode):
    params, st = perturbed_block(material=0)
    vals = inputs.fourier_wind(8, 2, seed=1)
    mpm = B.MPM.from_params(params, max_particles=st[0].shape[1], p2g_mode=mode)
    a = state_to_dev(st)
    out = B.MpmState.empty_like(a)
    mpm.substep(a, out, None, wind_dev(vals, 0.01), 0.0)
    b = state_to_dev(st)
    mpm.substep(b, b, None, wind_dev(vals, 0.01), 0.0)
    for u, w in zip(out, b):
        assert torch.allclose(u, w, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("material", [0, 1])
@pytest.mark.parametrize("mode", MODES)
def test_block_scene_100_substeps_positions_within_1e4(material, mode):
    """The forward block scene (32^3, 8192 particles, constant 5 N/kg wind,
    gravity, sticky walls, dt = 1e-4, 100 substeps), started from a perturbed
    state so that the constitutive model is exercised."""
    sc = inputs.block_scene()
    sc.material = material
    st = inputs.perturbed_state(sc.x, v_scale=0.2, c_scale=2.0, f_scale=0.02, seed=11)
    params = sc.params()
    mpm = B.MPM.from_params(params, max_particles=sc.n, p2g_mode=mode)
    s = state_to_dev(st)
    w = wind_dev(sc.wind, sc.t_total)
    for k in range(sc.n_substeps):
        mpm.substep(s, s, None, w, k * sc.dt)
    mpm.device_status()
    ref = oracle.mpm_rollout(params, f64(st), sc.wind_tuple(), 0.0, sc.n_substeps)
    g = state_to_np(s)
    assert np.abs(g[0] - ref[0]).max() <= 1e-4
    assert max_rel(g[3], ref[3]) <= 1e-4


def test_block_scene_rest_start_matches_closed_form():
    """From rest the block stays rigid: x_n = x_0 + dt^2 a n(n+1)/2."""
    sc = inputs.block_scene()
    st = inputs.rest_state(sc.x)
    mpm = B.MPM.from_params(sc.params(), max_particles=sc.n)
    s = state_to_dev(st)
    w = wind_dev(sc.wind, sc.t_total)
    for k in range(100):
        mpm.substep(s, s, None, w, k * sc.dt)
    a = np.array([5.0, -9.8, 0.0])
    expect = sc.x.astype(np.float64) + 1e-8 * a[:, None] * 5050
    assert np.abs(s.x.cpu().numpy() - expect).max() <= 1e-5


def test_sheet_full_size_three_substeps():
    """The flag-like sheet at full size (400,040 particles, 128^3, 32^3 x 16
    Fourier wind, pinned edge), three substeps from rest, all particles."""
    sc = inputs.sheet_scene()
    st = inputs.rest_state(sc.x)
    params = sc.params()
    mpm = B.MPM.from_params(params, max_particles=sc.n)
    s = state_to_dev(st)
    w = wind_dev(sc.wind, sc.t_total)
    pin = to_dev(sc.pinned)
    for k in range(3):
        mpm.substep(s, s, pin, w, k * sc.dt)
    mpm.device_status()
    ref = f64(st)
    for k in range(3):
        ref = oracle.mpm_substep(params, ref, sc.wind_tuple(), k * sc.dt, sc.pinned)
    check_state(s, ref, "sheet")


def test_out_of_domain_particle_sets_device_status():
    params, st = perturbed_block(material=0)
    x = st[0].copy()
    x[0, 5] = 0.01  # base index -1 on a 32^3 grid
    st = (x,) + st[1:]
    mpm = B.MPM.from_params(params, max_particles=x.shape[1])
    s = state_to_dev(st)
    mpm.substep(s, s, None, wind_dev(inputs.constant_wind(2, 1, (0, 0, 0)), 1.0), 0.0)
    with pytest.raises(B.DiffWindError, match="DW_ERR_DOMAIN"):
        mpm.device_status()
    mpm.device_status()  # cleared by the read
    assert s.x[0, 5].item() == pytest.approx(0.01)  # left unchanged


def test_empty_state_and_capacity_check():
    params, st = perturbed_block()
    mpm = B.MPM.from_params(params, max_particles=10)
    e = B.MpmState(*(torch.empty((r, 0), device="cuda") for r in (3, 3, 9, 9)))
    w = wind_dev(inputs.constant_wind(2, 1, (0, 0, 0)), 1.0)
    mpm.substep(e, e, None, w, 0.0)
    with pytest.raises(B.DiffWindError, match="DW_ERR_ARG"):
        big = state_to_dev(st)
        mpm.substep(big, big, None, w, 0.0)


# ------------------------------------------------------------------- sort --

def test_sort_is_a_permutation_by_cell_and_preserves_the_substep():
    params, st = perturbed_block(n_sub=10, material=1)
    n = st[0].shape[1]
    rng = np.random.default_rng(5)
    shuffle = rng.permutation(n)
    st = tuple(a[:, shuffle].copy() for a in st)
    pinned = (rng.random(n) < 0.2).astype(np.uint8)
    mpm = B.MPM.from_params(params, max_particles=n)
    a = state_to_dev(st)
    srt = B.MpmState.empty_like(a)
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    pin_s = torch.empty(n, dtype=torch.uint8, device="cuda")
    mpm.sort(a, srt, to_dev(pinned), pin_s, None, perm)
    p = perm.cpu().numpy()
    assert np.array_equal(np.sort(p), np.arange(n))
    for u, w in zip(srt, st):
        assert np.array_equal(u.cpu().numpy(), w[:, p])
    assert np.array_equal(pin_s.cpu().numpy(), pinned[p])
    # keys (4^3 block, then cell inside the block) are non-decreasing
    N = params["n_grid"]
    base = np.floor(st[0][:, p].astype(np.float64) * N - 0.5).astype(int)
    nb = (N + 3) // 4
    key = (((base[2] >> 2) * nb + (base[1] >> 2)) * nb + (base[0] >> 2)) * 64 + \
        ((base[2] & 3) * 4 + (base[1] & 3)) * 4 + (base[0] & 3)
    assert np.all(np.diff(key) >= 0)
    # a substep of the sorted state equals the permuted substep of the original
    vals = inputs.fourier_wind(8, 2, seed=9)
    w = wind_dev(vals, 0.01)
    out_a = B.MpmState.empty_like(a)
    mpm.substep(a, out_a, to_dev(pinned), w, 0.0)
    out_s = B.MpmState.empty_like(a)
    mpm.substep(srt, out_s, pin_s, w, 0.0)
    for u, v in zip(out_s, out_a):
        assert torch.allclose(u, v[:, perm.long()], rtol=1e-4, atol=1e-6)
    # ids carried through a second sort compose the permutations
    srt2 = B.MpmState.empty_like(a)
    ids2 = torch.empty_like(perm)
    pin2 = torch.empty_like(pin_s)
    mpm.sort(out_s, srt2, pin_s, pin2, perm, ids2)
    for u, v in zip(srt2, out_a):
        assert torch.equal(u, v[:, ids2.long()]) or torch.allclose(u, v[:, ids2.long()], rtol=1e-4, atol=1e-6)


# ---------------------------------------------------------------- adjoint --

@pytest.mark.parametrize("material", [0, 1])
@pytest.mark.parametrize("mode", [B.P2G_ATOMIC, B.P2G_TILE])
def test_substep_adjoint_matches_oracle(material, mode):
    params, st = perturbed_block(material=material, n_sub=6)
    n = st[0].shape[1]
    rng = np.random.default_rng(8)
    pinned = (rng.random(n) < 0.15).astype(np.uint8)
    vals = inputs.fourier_wind(8, 3, seed=5)
    g_out = tuple(rng.standard_normal(a.shape).astype(np.float32) for a in st)
    mpm = B.MPM.from_params(params, max_particles=n, p2g_mode=mode)
    g_in = B.MpmState.empty_like(state_to_dev(st))
    g_wind = torch.zeros(vals.shape, dtype=torch.float32, device="cuda")
    g_E = torch.zeros(1, dtype=torch.float32, device="cuda")
    mpm.substep_adjoint(state_to_dev(st), state_to_dev(g_out), g_in, to_dev(pinned),
                        wind_dev(vals, 0.01), 0.0031, g_wind, g_E)
    mpm.device_status()
    rg, rgw, rgE = oracle.mpm_substep_adjoint(params, f64(st), wind_ref(vals, 0.01), 0.0031,
                                              f64(g_out), pinned)
    for name, a, b in zip("xvCF", state_to_np(g_in), rg):
        assert rel_l2(a, b) <= 1e-4, (name, rel_l2(a, b))
    assert rel_l2(g_wind.cpu().numpy(), rgw) <= 1e-4
    assert abs(g_E.item() - rgE) <= 1e-4 * abs(rgE)


def test_adjoint_accumulates_and_may_alias_g_out():
    params, st = perturbed_block(material=0, n_sub=5)
    n = st[0].shape[1]
    rng = np.random.default_rng(3)
    g_out = tuple(rng.standard_normal(a.shape).astype(np.float32) for a in st)
    vals = inputs.fourier_wind(8, 2, seed=2)
    mpm = B.MPM.from_params(params, max_particles=n)
    w = wind_dev(vals, 0.01)
    g1 = B.MpmState.empty_like(state_to_dev(st))
    gw = torch.zeros(vals.shape, device="cuda")
    gE = torch.zeros(1, device="cuda")
    mpm.substep_adjoint(state_to_dev(st), state_to_dev(g_out), g1, None, w, 0.0, gw, gE)
    gw1, gE1 = gw.clone(), gE.clone()
    g2 = state_to_dev(g_out)
    mpm.substep_adjoint(state_to_dev(st), g2, g2, None, w, 0.0, gw, gE)  # in place, accumulate
    for a, b in zip(g1, g2):
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-6 * a.abs().max().item())
    assert torch.allclose(gw, 2 * gw1, rtol=1e-4, atol=1e-6 * gw1.abs().max().item())
    assert torch.allclose(gE, 2 * gE1, rtol=1e-4)


# ---------------------------------------------------------------- rollout --

@pytest.mark.parametrize("n_sub,sort_every", [(60, 20), (50, 20), (30, 0), (7, 3)])
def test_rollout_matches_oracle_and_substep_loop(n_sub, sort_every):
    """mpm_rollout (sorting + fused G2P/P2G) against the oracle and against the
    plain substep loop; ids map the sorted particles back."""
    sc = inputs.block_scene()
    rng = np.random.default_rng(3)
    st = inputs.perturbed_state(sc.x, v_scale=0.2, c_scale=2.0, f_scale=0.02, seed=5)
    shuffle = rng.permutation(sc.n)
    st = tuple(a[:, shuffle].copy() for a in st)
    pinned = (rng.random(sc.n) < 0.05).astype(np.uint8)
    vals = inputs.fourier_wind(8, 3, seed=4)
    params = sc.params()
    mpm = B.MPM.from_params(params, max_particles=sc.n)
    w = wind_dev(vals, n_sub * sc.dt)
    s = state_to_dev(st)
    pin = to_dev(pinned)
    ids = torch.arange(sc.n, dtype=torch.int32, device="cuda")
    mpm.rollout(s, pin, ids, w, 0.0, n_sub, sort_every)
    mpm.device_status()
    idx = ids.cpu().numpy()
    assert np.array_equal(np.sort(idx), np.arange(sc.n))
    assert np.array_equal(pin.cpu().numpy(), pinned[idx])
    ref = oracle.mpm_rollout(params, f64(st), wind_ref(vals, n_sub * sc.dt), 0.0, n_sub, pinned)
    g = state_to_np(s)
    assert np.abs(g[0] - ref[0][:, idx]).max() <= 1e-4
    assert max_rel(g[3], ref[3][:, idx]) <= 1e-4
    # the plain substep loop on the original order
    loop = state_to_dev(st)
    for k in range(n_sub):
        mpm.substep(loop, loop, to_dev(pinned), w, k * sc.dt)
    lp = state_to_np(loop)
    assert np.abs(g[0] - lp[0][:, idx]).max() <= 1e-5
    assert max_rel(g[1], lp[1][:, idx]) <= 1e-3


def test_rollout_sheet_full_size_positions_within_1e4():
    """The flag-like sheet at full size, 100 substeps through mpm_rollout with
    re-sorting every 15 (the bench's launch sequence), against the FP64 oracle
    on every particle."""
    sc = inputs.sheet_scene(n_substeps=100)
    params = sc.params()
    st = inputs.rest_state(sc.x)
    mpm = B.MPM.from_params(params, max_particles=sc.n)
    s = state_to_dev(st)
    pin = to_dev(sc.pinned)
    ids = torch.arange(sc.n, dtype=torch.int32, device="cuda")
    mpm.rollout(s, pin, ids, wind_dev(sc.wind, sc.t_total), 0.0, 100, 15)
    mpm.device_status()
    ref = oracle.mpm_rollout(params, f64(st), sc.wind_tuple(), 0.0, 100, sc.pinned)
    idx = ids.cpu().numpy()
    assert np.abs(s.x.cpu().numpy() - ref[0][:, idx]).max() <= 1e-4


@pytest.mark.parametrize("material", [0, 1])
@pytest.mark.parametrize("drop", [0, 1, 37])
@pytest.mark.parametrize("sort_every", [0, 10])
def test_rollout_fused_kernels_agree(material, drop, sort_every):
    """The two fused G2P/P2G kernels of mpm_rollout (two particles per thread
    on float2 pairs, P2G_PAIR; one particle per thread, P2G_WARP) against the
    FP64 oracle and against each other: both materials, an odd particle count
    (the scalar load path and a half-empty last pair), unsorted particles
    (sort_every = 0: warps span many cells, the grid-read G2P path, split
    pairs and the serial run walk) and sorted ones (staged G2P, one and two
    runs per warp), 5% pinned."""
    sc = inputs.block_scene()
    n = sc.n - drop
    rng = np.random.default_rng(11)
    st = inputs.perturbed_state(sc.x[:, :n], v_scale=0.2, c_scale=2.0, f_scale=0.02, seed=7)
    shuffle = rng.permutation(n)
    st = tuple(a[:, shuffle].copy() for a in st)
    pinned = (rng.random(n) < 0.05).astype(np.uint8)
    vals = inputs.fourier_wind(8, 3, seed=4)
    params = dict(sc.params(), material=material, E=1e4 if material else 3e4)
    n_sub = 30
    w = wind_dev(vals, n_sub * sc.dt)
    out = {}
    for mode in (B.P2G_PAIR, B.P2G_WARP):
        mpm = B.MPM.from_params(params, max_particles=n, p2g_mode=mode)
        s = state_to_dev(st)
        pin = to_dev(pinned)
        ids = torch.arange(n, dtype=torch.int32, device="cuda")
        mpm.rollout(s, pin, ids, w, 0.0, n_sub, sort_every)
        mpm.device_status()
        idx = ids.cpu().numpy()
        inv = np.empty(n, np.int64)
        inv[idx] = np.arange(n)
        out[mode] = tuple(a[:, inv] for a in state_to_np(s))  # back to the input order
        mpm.close()
    ref = oracle.mpm_rollout(params, f64(st), wind_ref(vals, n_sub * sc.dt), 0.0, n_sub, pinned)
    for mode, g in out.items():
        assert np.abs(g[0] - ref[0]).max() <= 1e-4, (mode, np.abs(g[0] - ref[0]).max())
        assert max_rel(g[3], ref[3]) <= 1e-4, (mode, max_rel(g[3], ref[3]))
    a, b = out[B.P2G_PAIR], out[B.P2G_WARP]
    assert np.abs(a[0] - b[0]).max() <= 1e-5
    assert max_rel(a[1], b[1]) <= 1e-3
    assert max_rel(a[3], b[3]) <= 1e-5


def test_rollout_pair_kernel_sheet_matches_one_per_thread():
    """The 400k-particle sheet (Neo-Hookean, 128^3, sorted every 20) through
    both fused kernels: positions within 1e-5 of each other after 60
    substeps, and every particle's deformation gradient within 1e-5."""
    sc = inputs.sheet_scene(n_substeps=60)
    params = sc.params()
    st = inputs.rest_state(sc.x)
    res = {}
    for mode in (B.P2G_PAIR, B.P2G_WARP):
        mpm = B.MPM.from_params(params, max_particles=sc.n, p2g_mode=mode)
        s = state_to_dev(st)
        pin = to_dev(sc.pinned)
        ids = torch.arange(sc.n, dtype=torch.int32, device="cuda")
        mpm.rollout(s, pin, ids, wind_dev(sc.wind, sc.t_total), 0.0, 60, 20)
        mpm.device_status()
        idx = ids.cpu().numpy()
        inv = np.empty(sc.n, np.int64)
        inv[idx] = np.arange(sc.n)
        res[mode] = (s.x.cpu().numpy()[:, inv], s.F.cpu().numpy()[:, inv])
        mpm.close()
    a, b = res[B.P2G_PAIR], res[B.P2G_WARP]
    assert np.abs(a[0] - b[0]).max() <= 1e-5
    assert np.abs(a[1] - b[1]).max() <= 1e-5
