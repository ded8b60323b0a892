"""The single-scene slab decomposition (paper_2603_09668_gb300.slab) on CPU:
two and three gloo ranks (127.0.0.1 rendezvous) each run the FP64 oracle's
P2G, grid update and G2P on their own particles of one tiny scene, joined by
the slab module's halo exchanges and particle migration, and must reproduce
the one-rank oracle substep by substep: the summed mass and momentum on every
owned node, the grid velocities in every layer a rank's stencils read, and the
final particle state (up to the order of the floating-point additions)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

N, N_SUB, SORT_EVERY, MARGIN = 16, 24, 6, 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def scene():
    from paper_2603_09668_gb300 import inputs

    x = inputs.block_particles(lo=(0.3, 0.3, 0.3), size=0.4, sub=6, per_sub=2, seed=11)
    x, v, C, F = inputs.perturbed_state(x, v_scale=0.3, c_scale=0.5, f_scale=0.01, seed=12)
    v = v.astype(np.float64)
    v[2] += 3.0 * np.sin(2 * np.pi * x[0])  # shear in z: particles cross the slab faces
    n = x.shape[1]
    params = dict(n_grid=N, dt=1e-3, gravity=(0.0, -9.8, 0.0), bc_band=2, material=0, E=1e3,
                  nu=0.3, p_mass=1000.0 * 0.4 ** 3 / n, p_vol=0.4 ** 3 / n)
    pinned = (np.random.default_rng(13).random(n) < 0.05).astype(np.float64)
    wind = (inputs.fourier_wind(4, 3, seed=14), 4, 3, N_SUB * params["dt"])
    state = tuple(np.asarray(a, np.float64) for a in (x, v, C, F))
    return params, state, pinned, wind


def _grid(gm, gp):
    return torch.from_numpy(np.concatenate([gm[None], gp])).view(4, N, N, N).clone()


def _rank(rank, world, port, out):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist

    import oracle
    from paper_2603_09668_gb300 import slab as SL

    dist.init_process_group("gloo", rank=rank, world_size=world)
    params, ref, pinned, wind = scene()
    sl = SL.Slab(N, world, rank, MARGIN)
    sl.validate()
    n = ref[0].shape[1]
    P = torch.from_numpy(np.concatenate(list(ref) + [pinned[None], np.arange(n, dtype=np.float64)[None]]))
    P = P[:, torch.from_numpy(sl.owner(ref[0][2]) == rank)]
    arrived = 0
    for k in range(N_SUB):
        t = k * params["dt"]
        if k and k % SORT_EVERY == 0:
            n_before = P.shape[1]
            kept = int((torch.from_numpy(sl.owner(P[2].numpy())) == rank).sum())
            P = SL.migrate(P, 2, sl)
            arrived += P.shape[1] - kept
            assert P.shape[1] - kept >= 0 and n_before >= kept
        sl.check_drift(P[2].numpy())
        x, v, C, F, pin = P[0:3].numpy(), P[3:6].numpy(), P[6:15].numpy(), P[15:24].numpy(), P[24].numpy()
        g = _grid(*oracle.mpm_p2g(params, x, v, C, F))
        nz = torch.nonzero(g.abs().sum(dim=(0, 2, 3))).flatten()
        assert nz.numel() == 0 or (int(nz.min()) >= sl.lo and int(nz.max()) < sl.hi)
        SL.halo_sum(g, sl)
        # one-rank reference of the same substep, stage by stage
        gm_r, gp_r = oracle.mpm_p2g(params, *ref)
        g_r = _grid(gm_r, gp_r)
        own = slice(sl.k0, sl.k1)
        scale = float(g_r.abs().max())
        assert float((g[:, own] - g_r[:, own]).abs().max()) <= 1e-12 * scale
        assert not g[:, :sl.k0].any() and not g[:, sl.k1:].any()
        gv = torch.from_numpy(oracle.mpm_grid_update(params, g[0].reshape(-1).numpy(),
                                                     g[1:].reshape(3, -1).numpy(), wind, t))
        gv = gv.view(3, N, N, N).clone()
        gv[:, :sl.k0] = 0
        gv[:, sl.k1:] = 0
        SL.halo_fill(gv, sl)
        gv_r = torch.from_numpy(oracle.mpm_grid_update(params, gm_r, gp_r, wind, t)).view(3, N, N, N)
        reach = slice(sl.lo, sl.hi)
        vscale = float(gv_r.abs().max())
        assert float((gv[:, reach] - gv_r[:, reach]).abs().max()) <= 1e-12 * vscale, k
        new = oracle.mpm_g2p(params, x, F, gv.reshape(3, -1).numpy(), pin)
        P = torch.from_numpy(np.concatenate(list(new) + [P[24:26].numpy()]))
        ref = oracle.mpm_g2p(params, ref[0], ref[3], gv_r.reshape(3, -1).numpy(), pinned)
    out[rank] = (P.numpy(), arrived)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_ranks_reproduce_the_one_rank_oracle(world):
    import oracle

    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == list(range(world))
    P = np.concatenate([res[r][0] for r in range(world)], axis=1)
    params, st, pinned, wind = scene()
    n = st[0].shape[1]
    assert P.shape[1] == n
    P = P[:, np.argsort(P[25])]
    assert np.array_equal(P[25], np.arange(n))  # every particle on exactly one rank
    ref = oracle.mpm_rollout(params, st, wind, 0.0, N_SUB, pinned.astype(np.uint8))
    for a, b, name in zip((P[0:3], P[3:6], P[6:15], P[15:24]), ref, "xvCF"):
        assert np.abs(a - b).max() <= 1e-9 * max(1.0, np.abs(b).max()), name
    assert sum(r[1] for r in res.values()) > 0  # particles did migrate between slabs


def test_slab_bounds_owner_and_drift_check():
    import sys

    sys.path.insert(0, ROOT)
    from paper_2603_09668_gb300 import slab as SL

    assert SL.layer_bounds(16, 3) == [0, 5, 10, 16]
    s = SL.Slab(16, 2, 0, margin=1)
    assert (s.k0, s.k1, s.lo, s.hi) == (0, 8, 0, 11)
    u = SL.Slab(16, 2, 1, margin=1)
    assert (u.k0, u.k1, u.lo, u.hi) == (8, 16, 7, 16)
    # base layer floor(16 z - 1/2): 7 -> rank 0, 8 -> rank 1
    z = (np.array([7, 8]) + 0.5 + 0.25) / 16
    assert list(s.owner(z)) == [0, 1]
    s.check_drift((np.array([8]) + 0.75) / 16)  # within the margin
    with pytest.raises(RuntimeError):
        s.check_drift((np.array([9]) + 0.75) / 16)
    with pytest.raises(RuntimeError):
        u.check_drift((np.array([6]) + 0.75) / 16)
    with pytest.raises(ValueError):
        SL.Slab(8, 4, 0, margin=1).validate()  # 2-layer slabs, 3-layer halo
