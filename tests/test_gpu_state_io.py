"""GPU tests of the host checkpoints of an MPM state (mpm_state_save,
mpm_state_peek, mpm_state_load): a save and a load reproduce the device
arrays bit for bit; a rollout stopped, saved, loaded into a new handle in
fresh buffers and resumed matches the uninterrupted rollout (to the float
atomics' summation order); wrong sizes and damaged files are errors."""
import numpy as np
import pytest
import torch

from paper_2603_09668_gb300 import binding as B
from paper_2603_09668_gb300 import inputs

from gpu_util import state_to_dev, state_to_np, to_dev, wind_dev

pytestmark = pytest.mark.gpu


def test_save_and_load_reproduce_the_state_bitwise(tmp_path):
    x = inputs.block_particles(sub=8, per_sub=2, seed=1)[:, :1001]  # an odd count
    st = state_to_dev(inputs.perturbed_state(x, v_scale=0.3, seed=2))
    n = st.n
    pin = to_dev((np.random.default_rng(3).random(n) < 0.1).astype(np.uint8))
    ids = torch.randperm(n, dtype=torch.int32, device="cuda")
    p = str(tmp_path / "a.dwst")
    B.mpm_state_save(p, st, pin, ids, t=0.0375, substep=750)
    assert B.mpm_state_peek(p) == dict(n=n, has_pinned=True, has_ids=True, t=0.0375, substep=750)
    out = B.MpmState.zeros_like(st)
    pin2 = torch.zeros_like(pin)
    ids2 = torch.zeros_like(ids)
    t, k = B.mpm_state_load(p, out, pin2, ids2)
    assert (t, k) == (0.0375, 750)
    for a, b in zip(out, st):
        assert torch.equal(a, b)
    assert torch.equal(pin2, pin) and torch.equal(ids2, ids)
    # the optional arrays may be left out on either side
    q = str(tmp_path / "b.dwst")
    B.mpm_state_save(q, st)
    out2 = B.MpmState.zeros_like(st)
    B.mpm_state_load(q, out2)
    assert torch.equal(out2.F, st.F)
    with pytest.raises(B.DiffWindError, match="DW_ERR_ARG"):
        B.mpm_state_load(q, out2, pinned=pin2)  # the file has no pinned array


def test_resumed_rollout_matches_the_uninterrupted_one(tmp_path):
    sc = inputs.sheet_scene(nu=80, nv=54, n_grid=64, n_substeps=100, dt=1e-4, wind_nf=16,
                            wind_frames=8, seed=0)
    params, n, dt = sc.params(), sc.n, sc.dt
    wind = wind_dev(sc.wind, sc.t_total)
    st0 = inputs.rest_state(sc.x)

    def run(state, pin, ids, t0, k):
        mpm = B.MPM.from_params(params, max_particles=n)
        mpm.rollout(state, pin, ids, wind, t0, k, 20)
        mpm.device_status()
        mpm.close()

    ref = state_to_dev(st0)
    ref_pin, ref_ids = to_dev(sc.pinned), torch.arange(n, dtype=torch.int32, device="cuda")
    run(ref, ref_pin, ref_ids, 0.0, 100)

    a = state_to_dev(st0)
    a_pin, a_ids = to_dev(sc.pinned), torch.arange(n, dtype=torch.int32, device="cuda")
    run(a, a_pin, a_ids, 0.0, 60)
    p = str(tmp_path / "roll.dwst")
    B.mpm_state_save(p, a, a_pin, a_ids, t=60 * dt, substep=60)
    del a, a_pin, a_ids
    hd = B.mpm_state_peek(p)
    b = B.MpmState(*(torch.empty((r, hd["n"]), device="cuda") for r in (3, 3, 9, 9)))
    b_pin = torch.empty(hd["n"], dtype=torch.uint8, device="cuda")
    b_ids = torch.empty(hd["n"], dtype=torch.int32, device="cuda")
    t, k = B.mpm_state_load(p, b, b_pin, b_ids)
    assert k == 60 and t == pytest.approx(60 * dt)
    run(b, b_pin, b_ids, t, 100 - k)

    def unsorted(s, ids):
        idx = ids.cpu().numpy()
        inv = np.empty(n, np.int64)
        inv[idx] = np.arange(n)
        return [a[:, inv] for a in state_to_np(s)]

    g, r = unsorted(b, b_ids), unsorted(ref, ref_ids)
    assert np.abs(g[0] - r[0]).max() <= 1e-5
    assert np.abs(g[3] - r[3]).max() <= 1e-5
    assert np.abs(g[0] - st0[0]).max() > 1e-4  # the sheet did move


def test_wrong_sizes_and_damaged_files_are_errors(tmp_path):
    x = inputs.block_particles(sub=4, per_sub=2, seed=4)
    st = state_to_dev(inputs.perturbed_state(x, seed=5))
    p = tmp_path / "c.dwst"
    B.mpm_state_save(str(p), st)
    small = B.MpmState(*(torch.zeros((r, st.n - 1), device="cuda") for r in (3, 3, 9, 9)))
    with pytest.raises(B.DiffWindError, match="DW_ERR_ARG"):
        B.mpm_state_load(str(p), small)
    data = p.read_bytes()
    short = tmp_path / "short.dwst"
    short.write_bytes(data[:-4])
    with pytest.raises(B.DiffWindError, match="DW_ERR_IO"):
        B.mpm_state_load(str(short), B.MpmState.zeros_like(st))
    long = tmp_path / "long.dwst"
    long.write_bytes(data + b"\0")
    with pytest.raises(B.DiffWindError, match="DW_ERR_IO"):
        B.mpm_state_load(str(long), B.MpmState.zeros_like(st))
    with pytest.raises(B.DiffWindError, match="DW_ERR_IO"):
        B.mpm_state_save(str(tmp_path / "no_such_dir" / "d.dwst"), st)
    assert not (tmp_path / "c.dwst.tmp").exists()
