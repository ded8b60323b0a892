"""mpm_substep_noalloc: the substep for callers that cannot allocate device
memory when they call (an allocator callback, a no-allocation real-time loop,
a host whose pool owns the device). It keeps its scratch grid in a fixed
device array inside the library instead of a handle's workspace.

These tests call it through the C-ABI and compare it with mpm_substep on the
same inputs, for two calls in a row, within the single-substep tolerances of
the MPM parity tests. This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from paper_2603_09668_gb300 import binding as B
from paper_2603_09668_gb300 import inputs

from gpu_util import max_rel, state_to_dev, state_to_np, to_dev, wind_dev

pytestmark = pytest.mark.gpu


def close(a, b):
    ga, gb = state_to_np(a), state_to_np(b)
    assert np.abs(ga[0] - gb[0]).max() <= 1e-6
    assert max_rel(ga[1], gb[1]) <= 1e-4
    assert max_rel(ga[2], gb[2]) <= 2e-3
    assert np.abs(ga[3] - gb[3]).max() <= 1e-6


@pytest.mark.parametrize("N,material", [(32, 1), (64, 0)])
def test_noalloc_matches_handle_substep_twice(N, material):
    x = inputs.block_particles(sub=10, per_sub=2, seed=4)
    st = inputs.perturbed_state(x, v_scale=0.05, c_scale=0.5, f_scale=0.01, seed=4)
    n = x.shape[1]
    params = dict(n_grid=N, dt=1e-4, gravity=(0.0, -9.8, 0.0), bc_band=3, material=material,
                  E=1e4, nu=0.3, p_mass=1000.0 * 0.25 ** 3 / n, p_vol=0.25 ** 3 / n)
    pinned = to_dev((np.random.default_rng(1).random(n) < 0.1).astype(np.uint8))
    wind = wind_dev(inputs.fourier_wind(8, 4, seed=3), 0.01)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")

    mpm = B.MPM.from_params(params, max_particles=n)
    ref = state_to_dev(st)
    got = state_to_dev(st)
    for call in range(2):
        t = call * params["dt"]
        ref_next = B.MpmState.empty_like(ref)
        mpm.substep(ref, ref_next, pinned, wind, t)
        got_next = B.MpmState.empty_like(got)
        B.mpm_substep_noalloc(params, got, got_next, pinned, wind, t, status)
        torch.cuda.synchronize()
        close(got_next, ref_next)
        ref, got = ref_next, got_next
    assert status.item() == 0
    mpm.device_status()
    mpm.close()


def test_noalloc_in_place_and_reports_device_errors():
    x = inputs.block_particles(sub=6, per_sub=2, seed=2)
    st = inputs.perturbed_state(x, seed=2)
    n = x.shape[1]
    params = dict(n_grid=32, dt=1e-4, gravity=(0.0, -9.8, 0.0), bc_band=3, material=0,
                  E=1e4, nu=0.3, p_mass=1e-3, p_vol=1e-6)
    wind = wind_dev(inputs.constant_wind(4, 1, (5.0, 0.0, 0.0)), 1.0)
    a = state_to_dev(st)
    b = state_to_dev(st)
    out = B.MpmState.empty_like(a)
    B.mpm_substep_noalloc(params, a, out, None, wind, 0.0)
    B.mpm_substep_noalloc(params, b, b, None, wind, 0.0)
    close(b, out)
    # a particle outside the grid is reported through the caller's status word
    xs = st[0].copy()
    xs[1, 3] = 0.005
    c = state_to_dev((xs,) + st[1:])
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.mpm_substep_noalloc(params, c, c, None, wind, 0.0, status)
    torch.cuda.synchronize()
    assert status.item() & 2


def test_noalloc_rejects_grids_beyond_its_fixed_array():
    x = inputs.block_particles(sub=4, per_sub=1)
    st = state_to_dev(inputs.rest_state(x))
    params = dict(n_grid=128, dt=1e-4, gravity=(0.0, -9.8, 0.0), bc_band=3, material=0,
                  E=1e4, nu=0.3, p_mass=1e-3, p_vol=1e-6)
    wind = wind_dev(inputs.constant_wind(2, 1, (0.0, 0.0, 0.0)), 1.0)
    with pytest.raises(B.DiffWindError, match="n_grid"):
        B.mpm_substep_noalloc(params, st, st, None, wind, 0.0)
