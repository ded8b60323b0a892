"""GPU tests of the batched MPM (many scenes, one launch per substep) through
the C-ABI.

Parity: every scene of a batch must match the same scene run alone through
mpm_rollout (same substeps, same re-sorting), particle by particle after the
carried ids undo both sorts. Both runs sum the P2G contributions with float
atomics in an unspecified order, so they agree to float32 rounding, not
bitwise: positions within 1e-6 (absolute, of the unit domain), F within
1e-6, v and C within 1e-4 of their largest magnitude. One small scene of the
batch is also checked against the FP64 oracle (positions within 1e-4).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_09668_gb300 import binding as B
from paper_2603_09668_gb300 import inputs

from gpu_util import f64, max_rel, rel_l2, state_to_np, to_dev, wind_dev, wind_ref

pytestmark = pytest.mark.gpu

DT = 5e-5


def small_scenes():
    """Uneven scenes: grids 32^3 / 64^3, blocks (fixed-corotated) and sheets
    (Neo-Hookean, pinned edge), 1 to ~13k particles (ragged last work item,
    a one-particle scene), each with its own wind."""
    out = []
    specs = [("block", 32, 8, 2), ("sheet", 64, 110, 60), ("block", 64, 5, 1),
             ("one", 32, 0, 0), ("sheet", 32, 40, 30), ("block", 32, 12, 3)]
    for s, (kind, N, a, b) in enumerate(specs):
        if kind == "block":
            x = inputs.block_particles(sub=a, per_sub=b, seed=s)
            pinned = np.zeros(x.shape[1], np.uint8)
            mat, E, vol = 1, 1e4, 0.25 ** 3 / x.shape[1]
        elif kind == "sheet":
            x, pinned = inputs.sheet_particles(a, b, seed=s)
            h = 0.6 / (a - 1)
            mat, E, vol = 0, 5e4, 0.6 * 0.4 * 2 * h / x.shape[1]
        else:
            x = np.array([[0.5], [0.45], [0.52]], np.float32)
            pinned = np.zeros(1, np.uint8)
            mat, E, vol = 0, 1e4, 1e-6
        st = inputs.perturbed_state(x, v_scale=0.1, c_scale=1.0, f_scale=0.01, seed=10 + s)
        params = dict(n_grid=N, dt=DT, gravity=(0.0, -9.8, 0.0), bc_band=3, material=mat, E=E,
                      nu=0.3, p_mass=1000.0 * vol, p_vol=vol)
        wind = inputs.fourier_wind(16, 8, seed=100 + s)
        out.append((params, st, pinned, wind))
    return out


def concat(scenes):
    st = tuple(np.ascontiguousarray(np.concatenate([sc[1][i] for sc in scenes], axis=1))
               for i in range(4))
    pin = np.concatenate([sc[2] for sc in scenes])
    return st, pin


def make_batch(scenes, t_total):
    winds = [wind_dev(sc[3], t_total) for sc in scenes]
    return B.MPMBatch([(sc[0], sc[1][0].shape[1], w) for sc, w in zip(scenes, winds)])


def dev_state(st):
    return B.MpmState(*(to_dev(np.asarray(a, np.float32)) for a in st))


def run_batch(scenes, n_sub, sort_every, config=None):
    st, pin = concat(scenes)
    batch = make_batch(scenes, n_sub * DT)
    if config is not None:
        batch.set_config(*config)
    s = dev_state(st)
    p = to_dev(pin)
    ids = torch.arange(batch.n, dtype=torch.int32, device="cuda")
    batch.rollout(s, p, ids, 0.0, n_sub, sort_every)
    batch.device_status()
    cfg = batch.config()
    return batch, state_to_np(s), p.cpu().numpy(), ids.cpu().numpy(), cfg


def unsort(arrs, idx):
    """Arrays in sorted order -> original order, given the carried ids."""
    out = []
    for a in arrs:
        b = np.empty_like(a)
        b[..., idx] = a
        out.append(b)
    return out


def assert_close(g, r, label, tol_xF=1e-6, tol_vC=1e-4):
    dx = np.abs(g[0] - r[0]).max()
    dF = np.abs(g[3] - r[3]).max()
    assert dx <= tol_xF, (label, "x", dx)
    assert dF <= tol_xF, (label, "F", dF)
    assert max_rel(g[1], r[1]) <= tol_vC, (label, "v", max_rel(g[1], r[1]))
    assert max_rel(g[2], r[2]) <= tol_vC, (label, "C", max_rel(g[2], r[2]))


# The paired kernel (BATCH_PAIR, the default) evaluates the same formulas in
# another order (paired sums, row-summed P2G) than the one-particle kernels of
# the other modes: across the two families x and F agree to 1e-5 and v, C to
# 1e-3 of their largest magnitude, as mpm_rollout's two fused kernels do.
CROSS = dict(tol_xF=1e-5, tol_vC=1e-3)


@pytest.mark.parametrize("sort_every", [0, 7])
def test_each_scene_matches_the_scene_run_alone(sort_every):
    scenes = small_scenes()
    n_sub = 24
    batch, g, gpin, gids, cfg = run_batch(scenes, n_sub, sort_every)
    assert cfg["mode"] == B.BATCH_PAIR  # the default
    for s, (params, st, pinned, wind) in enumerate(scenes):
        sl = batch.scene_slice(s)
        n = st[0].shape[1]
        local = gids[sl] - batch.offsets[s]
        assert np.array_equal(np.sort(local), np.arange(n)), s  # a permutation within the scene
        assert np.array_equal(gpin[sl], pinned[local])
        mine = unsort([a[:, sl] for a in g], local)
        mpm = B.MPM.from_params(params, max_particles=n)
        a = dev_state(st)
        ids = torch.arange(n, dtype=torch.int32, device="cuda")
        mpm.rollout(a, to_dev(pinned), ids, wind_dev(wind, n_sub * DT), 0.0, n_sub, sort_every)
        mpm.device_status()
        alone = unsort(list(state_to_np(a)), ids.cpu().numpy())
        assert_close(mine, alone, f"scene {s}")
        mpm.close()
    batch.close()


def test_batch_scene_matches_oracle():
    scenes = small_scenes()
    n_sub = 20
    batch, g, _, gids, _ = run_batch(scenes, n_sub, 10)
    s = 0
    params, st, pinned, wind = scenes[s]
    sl = batch.scene_slice(s)
    mine = unsort([a[:, sl] for a in g], gids[sl] - batch.offsets[s])
    ref = oracle.mpm_rollout(params, f64(st), wind_ref(wind, n_sub * DT), 0.0, n_sub, pinned)
    assert np.abs(mine[0] - ref[0]).max() <= 1e-4
    assert np.abs(mine[3] - ref[3]).max() <= 1e-4
    batch.close()


@pytest.mark.parametrize("config", [(B.BATCH_PERSISTENT, 256, 1, 1), (B.BATCH_PERSISTENT, 128, 2, 0),
                                    (B.BATCH_SPLIT, 128, 4, 1), (B.BATCH_SPLIT, 256, 2, 0),
                                    (B.BATCH_PAIR, 256, 2, 1), (B.BATCH_PAIR, 128, 4, 0)])
def test_launch_shapes_agree(config):
    scenes = small_scenes()
    n_sub = 16
    b0, g0, _, ids0, _ = run_batch(scenes, n_sub, 5)
    b1, g1, _, ids1, cfg = run_batch(scenes, n_sub, 5, config)
    assert cfg["mode"] == config[0] and cfg["threads"] == config[1]
    tol = {} if config[0] == B.BATCH_PAIR else CROSS  # the default is BATCH_PAIR
    assert_close(unsort(list(g1), ids1), unsort(list(g0), ids0), str(config), **tol)
    b0.close()
    b1.close()


def test_pair_mode_vector_loads_match_split_mode():
    """Scenes of multiples of 4 particles: the pair kernel loads x and F as
    float2 and 16-byte pieces (every work item starts 16-byte aligned). Each
    scene must match split mode (one particle per thread), with re-sorts and
    both materials; the scenes end in work items of 16, 124 (64 + 60), 96
    (64 + 32) and 64 particles (a warp with none)."""
    scenes = []
    for params, st, pinned, wind in small_scenes():
        n = st[0].shape[1] - st[0].shape[1] % 4
        if n == 0:
            continue
        scenes.append((params, tuple(np.ascontiguousarray(a[:, :n]) for a in st), pinned[:n], wind))
    assert all(sc[1][0].shape[1] % 4 == 0 for sc in scenes)
    assert {sc[0]["material"] for sc in scenes} == {0, 1}
    n_sub = 24
    b0, g0, _, ids0, cfg0 = run_batch(scenes, n_sub, 7, (B.BATCH_PAIR, 128, 4, 1))
    b1, g1, _, ids1, cfg1 = run_batch(scenes, n_sub, 7, (B.BATCH_SPLIT, 128, 4, 1))
    assert cfg0["mode"] == B.BATCH_PAIR and cfg1["mode"] == B.BATCH_SPLIT
    assert_close(unsort(list(g0), ids0), unsort(list(g1), ids1), "pair vs split", **CROSS)
    b0.close()
    b1.close()


def test_graph_replay_repeats_and_time_advances():
    """A graph is captured once per rollout shape: two rollouts of 8 substeps
    from t0 = 0 and t0 = 8 dt equal one eager rollout of 16 (wind varies in
    time, so a stale t0 would show)."""
    scenes = small_scenes()
    st, pin = concat(scenes)
    batch = make_batch(scenes, 16 * DT)
    s = dev_state(st)
    p = to_dev(pin)
    batch.rollout(s, p, None, 0.0, 8, 0)
    batch.rollout(s, p, None, 8 * DT, 8, 0)
    batch.device_status()
    assert batch.config()["graph_active"] == 1
    eager = make_batch(scenes, 16 * DT)
    eager.set_config(B.BATCH_PAIR, 128, 4, use_graph=0)
    e = dev_state(st)
    eager.rollout(e, to_dev(pin), None, 0.0, 16, 0)
    eager.device_status()
    assert eager.config()["graph_active"] == 0
    assert_close(list(state_to_np(s)), list(state_to_np(e)), "graph vs eager")
    batch.close()
    eager.close()


def test_autotuner_picks_a_measured_candidate_and_leaves_state():
    scenes = small_scenes()
    st, pin = concat(scenes)
    batch = make_batch(scenes, 10 * DT)
    s = dev_state(st)
    p = to_dev(pin)
    before = [a.clone() for a in s]
    best, trials = batch.tune(s, p, n_trial_substeps=5)
    assert len(trials) >= 4
    assert {t[0]["mode"] for t in trials} == {B.BATCH_PERSISTENT, B.BATCH_SPLIT, B.BATCH_PAIR}
    fastest = min(trials, key=lambda t: t[1])
    assert {k: best[k] for k in ("mode", "threads", "ctas_per_sm")} == \
        {k: fastest[0][k] for k in ("mode", "threads", "ctas_per_sm")}
    assert all(t[1] > 0 for t in trials)
    for a, b in zip(s, before):
        assert torch.equal(a, b)
    cfg = batch.config()
    assert cfg["mode"] == best["mode"] and cfg["threads"] == best["threads"]
    batch.rollout(s, p, None, 0.0, 4, 0)  # the tuned configuration runs
    batch.device_status()
    batch.close()


def test_barrier_wait_is_bounded_and_reports_timeout():
    """The grid barrier told to wait for CTAs that were never launched gives
    up after its bounded wait and reports DW_ERR_TIMEOUT; the batch works
    afterwards."""
    scenes = small_scenes()[:2]
    batch = make_batch(scenes, 4 * DT)
    batch.barrier_selftest(0)
    with pytest.raises(B.DiffWindError) as ei:
        batch.barrier_selftest(1)
    assert ei.value.status == 6  # DW_ERR_TIMEOUT
    st, pin = concat(scenes)
    s = dev_state(st)
    batch.rollout(s, to_dev(pin), None, 0.0, 4, 0)
    batch.device_status()
    assert np.isfinite(state_to_np(s)[0]).all()
    batch.close()


def test_domain_error_is_reported_per_batch():
    scenes = small_scenes()[:3]
    scenes[1][1][0][:, 0] = (0.999, 0.5, 0.5)  # a particle outside the stencil range
    st, pin = concat(scenes)
    batch = make_batch(scenes, 2 * DT)
    s = dev_state(st)
    batch.rollout(s, to_dev(pin), None, 0.0, 2, 0)
    with pytest.raises(B.DiffWindError) as ei:
        batch.device_status()
    assert ei.value.status == 5  # DW_ERR_DOMAIN
    batch.device_status()  # cleared
    batch.close()


# ---------------------------------------------------------------- reverse --

def batch_adjoint(scenes, n_sub, g_seed=4):
    """mpm_batch_segment_adjoint over n_sub substeps from the scenes' states
    with a random dL/d(final state): (batch, gradient state, g_wind, g_E,
    the seed gradient, the tape)."""
    st, pin = concat(scenes)
    batch = make_batch(scenes, n_sub * DT)
    rng = np.random.default_rng(g_seed)
    g_out = tuple(rng.standard_normal(a.shape).astype(np.float32) for a in st)
    g = dev_state(g_out)
    nw, _ = batch.wind_layout()
    g_wind = torch.zeros(nw, dtype=torch.float32, device="cuda")
    g_E = torch.zeros(len(scenes), dtype=torch.float32, device="cuda")
    tape = torch.empty(max(n_sub - 1, 1) * 24 * batch.n, dtype=torch.float32, device="cuda")
    batch.segment_adjoint(dev_state(st), tape, g, to_dev(pin), 0.0, n_sub, g_wind, g_E)
    batch.device_status()
    return batch, state_to_np(g), g_wind.cpu().numpy(), g_E.cpu().numpy(), g_out, tape


def test_wind_layout_concatenates_the_scenes_wind_values():
    scenes = small_scenes()
    batch = make_batch(scenes, DT)
    total, offs = batch.wind_layout()
    sizes = [sc[3].size for sc in scenes]
    assert offs == [int(v) for v in np.concatenate([[0], np.cumsum(sizes)])]
    assert total == sum(sizes)
    batch.close()


@pytest.mark.parametrize("p2g_mode", [B.P2G_WARP, B.P2G_AUTO])
def test_batch_segment_adjoint_matches_each_scene_alone(p2g_mode):
    """Every scene's gradients (state, wind, E) from one batched segment
    adjoint equal those of mpm_segment_adjoint on the scene alone, and the
    batched tape holds the same recomputed states. The batched recompute runs
    the one-particle-per-thread substep kernels: against the single-scene
    adjoint with the same kernels (P2G_WARP) the results agree up to the
    float atomics' summation order (relative L2 1e-4); against the
    single-scene default (P2G_AUTO: the recompute on the paired kernel, whose
    FFMA2 products round differently) the 10 recomputed substeps differ by
    the cross-kernel rounding of the forward tests (1e-5 in x), which the
    reverse pass carries into the gradients at up to a few 1e-4 (bound 1e-3)."""
    tol = 1e-4 if p2g_mode == B.P2G_WARP else 1e-3
    scenes = small_scenes()
    n_sub = 10
    batch, gb, gw, gE, g_out, tape = batch_adjoint(scenes, n_sub)
    _, woff = batch.wind_layout()
    n = batch.n
    tape_np = tape.cpu().numpy()
    for s, (params, st, pinned, wind) in enumerate(scenes):
        sl = batch.scene_slice(s)
        ns = st[0].shape[1]
        mpm = B.MPM.from_params(params, max_particles=ns, p2g_mode=p2g_mode)
        g = dev_state(tuple(a[:, sl] for a in g_out))
        gw_s = torch.zeros(wind.size, dtype=torch.float32, device="cuda")
        gE_s = torch.zeros(1, dtype=torch.float32, device="cuda")
        tape_s = torch.empty((n_sub - 1) * 24 * ns, dtype=torch.float32, device="cuda")
        mpm.segment_adjoint(dev_state(st), tape_s, g, to_dev(pinned), wind_dev(wind, n_sub * DT),
                            0.0, n_sub, gw_s, gE_s)
        mpm.device_status()
        ref = state_to_np(g)
        for name, a, b in zip("xvCF", gb, ref):
            assert rel_l2(a[:, sl], b) <= tol, (s, name, rel_l2(a[:, sl], b))
        assert rel_l2(gw[woff[s]:woff[s + 1]], gw_s.cpu().numpy().ravel()) <= tol, s
        assert abs(gE[s] - gE_s.item()) <= tol * abs(gE_s.item()) + 1e-12, (s, gE[s], gE_s.item())
        # the last recomputed state of the segment, scene s's columns
        last = tape_np[(n_sub - 2) * 24 * n:(n_sub - 1) * 24 * n].reshape(24, n)[:, sl]
        last_s = tape_s.cpu().numpy()[(n_sub - 2) * 24 * ns:].reshape(24, ns)
        x_tol = 1e-6 if p2g_mode == B.P2G_WARP else CROSS["tol_xF"]
        assert np.abs(last[0:3] - last_s[0:3]).max() <= x_tol, s  # positions
        mpm.close()
    batch.close()


def test_batch_segment_adjoint_matches_oracle():
    """One block scene (fixed-corotated) and one pinned sheet scene
    (Neo-Hookean) of the batch against the FP64 oracle's reverse mode of the
    same 6 substeps (forward states recomputed by the oracle)."""
    scenes = small_scenes()
    n_sub = 6
    batch, gb, gw, gE, g_out, _ = batch_adjoint(scenes, n_sub, g_seed=9)
    _, woff = batch.wind_layout()
    for s in (0, 4):
        params, st, pinned, wind = scenes[s]
        sl = batch.scene_slice(s)
        w = wind_ref(wind, n_sub * DT)
        states = [f64(st)]
        for k in range(n_sub - 1):
            states.append(oracle.mpm_substep(params, states[-1], w, k * DT, pinned))
        g = tuple(np.asarray(a[:, sl], np.float64) for a in g_out)
        g_wind = np.zeros(wind.shape)
        g_E = 0.0
        for k in reversed(range(n_sub)):
            g, g_wind, e = oracle.mpm_substep_adjoint(params, states[k], w, k * DT, g, pinned,
                                                      g_wind)
            g_E += e
        for name, a, b in zip("xvCF", gb, g):
            assert rel_l2(a[:, sl], b) <= 1e-4, (s, name, rel_l2(a[:, sl], b))
        assert rel_l2(gw[woff[s]:woff[s + 1]], g_wind.ravel()) <= 1e-4, s
        assert abs(gE[s] - g_E) <= 1e-4 * abs(g_E), (s, gE[s], g_E)
    batch.close()


def test_batch_segment_adjoint_edge_cases():
    """One substep needs no tape; a short tape is rejected before any launch;
    gradients accumulate into g_wind and g_E across calls."""
    scenes = small_scenes()[:3]
    st, pin = concat(scenes)
    batch = make_batch(scenes, 4 * DT)
    nw, _ = batch.wind_layout()
    g_wind = torch.zeros(nw, device="cuda")
    g_E = torch.zeros(3, device="cuda")
    rng = np.random.default_rng(1)
    g_out = tuple(rng.standard_normal(a.shape).astype(np.float32) for a in st)
    g1 = dev_state(g_out)
    batch.segment_adjoint(dev_state(st), None, g1, to_dev(pin), 0.0, 1, g_wind, g_E)
    batch.device_status()
    gw1, gE1 = g_wind.clone(), g_E.clone()
    g2 = dev_state(g_out)
    batch.segment_adjoint(dev_state(st), None, g2, to_dev(pin), 0.0, 1, g_wind, g_E)
    batch.device_status()
    for a, b in zip(g1, g2):
        assert torch.allclose(a, b, rtol=1e-4, atol=1e-6 * a.abs().max().item())
    assert torch.allclose(g_wind, 2 * gw1, rtol=1e-4, atol=1e-6 * gw1.abs().max().item())
    assert torch.allclose(g_E, 2 * gE1, rtol=1e-4, atol=1e-12)
    short = torch.empty(24 * batch.n - 1, device="cuda")
    with pytest.raises(B.DiffWindError) as ei:
        batch.segment_adjoint(dev_state(st), short, dev_state(g_out), to_dev(pin), 0.0, 2)
    assert ei.value.status == 1  # DW_ERR_ARG
    batch.close()


def test_batch_segment_adjoint_graph_replay_equals_eager():
    """Two segments with different start states through the captured graph
    (the second a replay reading its start from the workspace) equal the
    same two segments launched eagerly."""
    scenes = small_scenes()[:4]
    st, pin = concat(scenes)
    st2 = tuple(a.copy() for a in st)
    st2[0][:] += np.float32(1e-3)  # a shifted start state for the second segment
    n_sub = 5
    rng = np.random.default_rng(12)
    g_out = tuple(rng.standard_normal(a.shape).astype(np.float32) for a in st)
    results = []
    for use_graph in (1, 0):
        batch = make_batch(scenes, 2 * n_sub * DT)
        batch.set_config(B.BATCH_PERSISTENT, 128, 1, use_graph)
        nw, _ = batch.wind_layout()
        g_wind = torch.zeros(nw, device="cuda")
        g_E = torch.zeros(len(scenes), device="cuda")
        tape = torch.empty((n_sub - 1) * 24 * batch.n, device="cuda")
        g = dev_state(g_out)
        p = to_dev(pin)
        batch.segment_adjoint(dev_state(st2), tape, g, p, n_sub * DT, n_sub, g_wind, g_E)
        batch.segment_adjoint(dev_state(st), tape, g, p, 0.0, n_sub, g_wind, g_E)
        batch.device_status()
        results.append((state_to_np(g), g_wind.cpu().numpy(), g_E.cpu().numpy()))
        batch.close()
    (ga, wa, ea), (gb, wb, eb) = results
    for name, a, b in zip("xvCF", ga, gb):
        assert rel_l2(a, b) <= 1e-5, (name, rel_l2(a, b))
    assert rel_l2(wa, wb) <= 1e-5
    assert np.allclose(ea, eb, rtol=1e-5, atol=1e-12)
