"""GPU tests of the checkpointed MPM autograd wrapper (autograd.mpm_frames):
segments run forward by mpm_rollout, reverse by mpm_segment_adjoint, with the
particles sorted by cell once at the start. Gradients of a random linear loss
on the checkpoint frames with respect to the wind values, E and the initial
state are compared with the FP64 oracle's reverse pass over the same substeps
(relative L2 2e-3: 24 float32 substeps forward and back in three chained
segments; the per-segment test in test_gpu_adjoint_segments.py measures how
the reverse pass's error grows, about 1.1e-5 per substep for dL/dx and far
less for every other block, so 24 substeps stay below 5e-4), and the sorted
and unsorted orders must agree (1e-4)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2603_09668_gb300 import autograd as AG
from paper_2603_09668_gb300 import binding as B
from paper_2603_09668_gb300 import inputs

from gpu_util import f64, rel_l2, to_dev, wind_ref

pytestmark = pytest.mark.gpu

N_SUB, EVERY = 24, 8


def setup(seed=3):
    x = inputs.block_particles(sub=8, per_sub=2, seed=seed)
    st = inputs.perturbed_state(x, v_scale=0.05, c_scale=0.5, f_scale=0.01, seed=seed)
    params = dict(n_grid=32, dt=1e-4, gravity=(0.0, -9.8, 0.0), bc_band=3, material=0, E=1e4,
                  nu=0.3, p_mass=1000.0 * 0.25 ** 3 / x.shape[1], p_vol=0.25 ** 3 / x.shape[1])
    rng = np.random.default_rng(seed)
    pinned = (rng.random(x.shape[1]) < 0.05).astype(np.uint8)
    vals = inputs.fourier_wind(8, 3, seed=seed + 1)
    weights = rng.standard_normal((N_SUB // EVERY, 3, x.shape[1]))
    return params, st, pinned, vals, weights


def gpu_grads(params, st, pinned, vals, weights, sort):
    mpm = B.MPM.from_params(params, max_particles=st[0].shape[1])
    s0 = B.MpmState(*(to_dev(np.asarray(a, np.float32)) for a in st))
    for a in s0:
        a.requires_grad_(True)
    wv = to_dev(vals.astype(np.float32)).requires_grad_(True)
    E = torch.tensor(params["E"], device="cuda", requires_grad=True)
    X = AG.mpm_frames(mpm, s0, wv, N_SUB * params["dt"], E, N_SUB, EVERY, pinned=to_dev(pinned),
                      sort=sort)
    loss = (X * to_dev(weights.astype(np.float32))).sum()
    loss.backward()
    mpm.device_status()
    out = {"wind": wv.grad.double().cpu().numpy(), "E": float(E.grad), "x0": s0.x.grad.double().cpu().numpy(),
           "F0": s0.F.grad.double().cpu().numpy(), "X": X.detach().double().cpu().numpy()}
    mpm.close()
    return out


def oracle_grads(params, st, pinned, vals, weights):
    dt = params["dt"]
    w = wind_ref(vals, N_SUB * dt)
    states = [f64(st)]
    for k in range(N_SUB):
        states.append(oracle.mpm_substep(params, states[-1], w, k * dt, pinned))
    g = [np.zeros_like(a) for a in states[0]]
    g_wind = np.zeros(np.asarray(vals).shape)
    g_E = 0.0
    for k in reversed(range(N_SUB)):
        if (k + 1) % EVERY == 0:
            g[0] = g[0] + weights[(k + 1) // EVERY - 1]
        gi, g_wind, gE = oracle.mpm_substep_adjoint(params, states[k], w, k * dt, tuple(g), pinned,
                                                    g_wind)
        g = list(gi)
        g_E += gE
    frames = np.stack([states[EVERY * (f + 1)][0] for f in range(N_SUB // EVERY)])
    return {"wind": g_wind, "E": g_E, "x0": g[0], "F0": g[3], "X": frames}


def test_checkpointed_gradients_match_oracle():
    params, st, pinned, vals, weights = setup()
    gpu = gpu_grads(params, st, pinned, vals, weights, sort=True)
    ref = oracle_grads(params, st, pinned, vals, weights)
    assert np.abs(gpu["X"] - ref["X"]).max() <= 1e-5
    for k in ("wind", "x0", "F0"):
        assert rel_l2(gpu[k], ref[k]) <= 2e-3, (k, rel_l2(gpu[k], ref[k]))
    assert abs(gpu["E"] - ref["E"]) <= 2e-3 * abs(ref["E"]), (gpu["E"], ref["E"])


def test_sorted_and_unsorted_orders_agree():
    params, st, pinned, vals, weights = setup(seed=5)
    a = gpu_grads(params, st, pinned, vals, weights, sort=True)
    b = gpu_grads(params, st, pinned, vals, weights, sort=False)
    assert np.abs(a["X"] - b["X"]).max() <= 1e-6
    for k in ("wind", "x0", "F0"):
        assert rel_l2(a[k], b[k]) <= 1e-4, (k, rel_l2(a[k], b[k]))
    assert abs(a["E"] - b["E"]) <= 1e-4 * abs(b["E"])


def test_checkpointed_wind_and_E_gradients_match_central_differences():
    """The setting of the adjoint workload at a size the FP64 oracle finishes
    in seconds: a pinned Neo-Hookean sheet (40 x 27 x 2 particles, 32^3 grid,
    8^3 x 4 Fourier wind), 100 substeps with checkpoints every 25, loss
    L = (1/N) sum over the checkpoint frames and particles of |x - x_target|^2
    with the target trajectory driven by another wind field. The GPU
    gradients (checkpointed forward + mpm_segment_adjoint through
    autograd.mpm_frames) of 16 random wind entries among those the loss
    depends on, and of E, against central differences of the oracle's loss
    (eps = 1e-3 on a wind value, 1e-4 E on E): within 1e-2. The oracle's own
    reverse pass meets these differences to 1e-6, so the check measures the
    float32 path."""
    n_sub, every = 100, 25
    sc = inputs.sheet_scene(nu=40, nv=27, n_grid=32, n_substeps=n_sub, dt=1e-4, wind_nf=8,
                            wind_frames=4, seed=0, wind_seed=0)
    params, pinned = sc.params(), sc.pinned
    st = inputs.rest_state(sc.x)
    n = sc.n
    w_true = inputs.fourier_wind(8, 4, seed=77)
    t_total = n_sub * sc.dt

    def oracle_frames(vals, p=params):
        _, kept = oracle.mpm_rollout(p, f64(st), wind_ref(vals, t_total), 0.0, n_sub, pinned,
                                     keep_every=every)
        return np.stack([k[0] for k in kept[1:]])

    target = oracle_frames(w_true)

    def oracle_loss(vals, p=params):
        return float(((oracle_frames(vals, p) - target) ** 2).sum() / n)

    mpm = B.MPM.from_params(params, max_particles=n)
    s0 = B.MpmState(*(to_dev(np.asarray(a, np.float32)) for a in st))
    wv = to_dev(sc.wind.astype(np.float32)).requires_grad_(True)
    E = torch.tensor(params["E"], device="cuda", requires_grad=True)
    X = AG.mpm_frames(mpm, s0, wv, t_total, E, n_sub, every, pinned=to_dev(pinned))
    loss = ((X - to_dev(target.astype(np.float32))) ** 2).sum() / n
    loss.backward()
    mpm.device_status()
    g_wind = wv.grad.double().cpu().numpy().ravel()
    g_E = float(E.grad)
    mpm.close()

    # entries the loss depends on: the oracle adjoint's nonzero wind gradient
    ref = oracle_grads_loss(params, st, pinned, sc.wind, target, n_sub, every, t_total)
    live = np.flatnonzero(np.abs(ref) > 1e-2 * np.abs(ref).max())
    pick = np.random.default_rng(0).choice(live, size=16, replace=False)
    eps = 1e-3
    fd = []
    for idx in pick:
        vp = np.asarray(sc.wind, np.float64).copy().ravel()
        vm = vp.copy()
        vp[idx] += eps
        vm[idx] -= eps
        fd.append((oracle_loss(vp.reshape(sc.wind.shape)) - oracle_loss(vm.reshape(sc.wind.shape)))
                  / (2 * eps))
    fd = np.array(fd)
    scale = np.abs(fd).max()
    err = np.abs(g_wind[pick] - fd) / np.maximum(np.abs(fd), 0.1 * scale)
    assert err.max() <= 1e-2, (err.max(), g_wind[pick], fd)
    eE = 1e-4 * params["E"]
    pp, pm = dict(params), dict(params)
    pp["E"] += eE
    pm["E"] -= eE
    fd_E = (oracle_loss(sc.wind, pp) - oracle_loss(sc.wind, pm)) / (2 * eE)
    assert abs(g_E - fd_E) <= 1e-2 * abs(fd_E), (g_E, fd_E)


def oracle_grads_loss(params, st, pinned, vals, target, n_sub, every, t_total):
    """dL/d(wind values) of the target-trajectory loss by the oracle's reverse
    pass (flattened)."""
    dt = params["dt"]
    w = wind_ref(vals, t_total)
    states = [f64(st)]
    for k in range(n_sub):
        states.append(oracle.mpm_substep(params, states[-1], w, k * dt, pinned))
    n = states[0][0].shape[1]
    g = [np.zeros_like(a) for a in states[0]]
    g_wind = np.zeros(np.asarray(vals).shape)
    for k in reversed(range(n_sub)):
        if (k + 1) % every == 0:
            f = (k + 1) // every - 1
            g[0] = g[0] + 2.0 * (states[k + 1][0] - target[f]) / n
        gi, g_wind, _ = oracle.mpm_substep_adjoint(params, states[k], w, k * dt, tuple(g), pinned,
                                                   g_wind)
        g = list(gi)
    return g_wind.ravel()
