"""CPU check of the HOME-LBM kernel's tiling: the kernel's own device
functions, compiled for the host (tests/home_tile_emulator.cu), run block by
block in the kernel's phase order and must match the FP64 oracle to float32
rounding on lattices with ragged tiles on every axis, several z ranges per
column, periodic and inlet/outlet boundaries, obstacles and forces. The
compact all-directions rebuild must equal the per-direction one."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2603_09668_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def emulator(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("emu") / "home_tile_emulator")
    csrc = os.path.join(ROOT, "paper_2603_09668_gb300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"), "-I", csrc,
                    "-gencode", "arch=compute_103a,code=sm_103a",
                    os.path.join(ROOT, "tests", "home_tile_emulator.cu"),
                    os.path.join(csrc, "status.cu"), "-o", exe], check=True,
                   capture_output=True)
    return exe


def test_compact_rebuild_equals_per_direction(emulator):
    out = subprocess.run([emulator, "rebuild-check"], check=True, capture_output=True, text=True)
    assert float(out.stdout) < 1e-6


@pytest.mark.parametrize("shape,tau,u_in,force,bc_x,steps,frac,tz", [
    ((16, 12, 10), 0.6, (0.05, 0.02, 0.0), (1e-5, -2e-5, 0.0), 1, 9, 0.1, 5),
    ((20, 9, 7), 0.8, (0.0, 0.0, 0.0), (0.0, 0.0, 3e-5), 0, 12, 0.0, 3),
    ((40, 17, 35), 0.55, (0.05, 0.0, 0.0), (0.0, 0.0, 0.0), 1, 3, 0.15, 8),
    ((33, 8, 16), 0.7, (0.03, 0.0, 0.01), (0.0, 0.0, 0.0), 0, 4, 0.05, 16),
])
def test_tiles_match_oracle(emulator, tmp_path, shape, tau, u_in, force, bc_x, steps, frac, tz):
    rng = np.random.default_rng(22)
    nc = int(np.prod(shape))
    m = oracle.home_init(shape, 1.0, (0.04, 0.01, 0.0), tau, force)
    m[0] += 2e-3 * rng.standard_normal(nc)
    m[1:4] += 1e-2 * rng.standard_normal((3, nc))
    m[4:] += 1e-4 * rng.standard_normal((6, nc))
    dev = m.copy()
    dev[0] -= 1.0
    dev = dev.astype(np.float32)
    ref = dev.astype(np.float64)
    ref[0] += 1.0
    fin, fout, fsol = tmp_path / "in.bin", tmp_path / "out.bin", tmp_path / "solid.bin"
    dev.tofile(fin)
    args = [emulator, *map(str, shape), str(tau), *map(str, u_in), *map(str, force), str(bc_x),
            str(steps), str(fin), str(fout)]
    solid = None
    if frac > 0:
        solid = inputs.random_mask(shape, frac, seed=21)
        solid.tofile(fsol)
        args += [str(fsol), str(tz)]
    subprocess.run(args, check=True)
    out = np.fromfile(fout, np.float32).reshape(10, -1).astype(np.float64)
    out[0] += 1.0
    refo = oracle.home_step(shape, tau, ref, steps, u_in=u_in, force=force, bc_x=bc_x, solid=solid)
    fl = np.ones(nc, bool) if solid is None else solid == 0
    _, u = oracle.home_macroscopic(shape, out, force, solid)
    _, ur = oracle.home_macroscopic(shape, refo, force, solid)
    assert np.linalg.norm(u[:, fl] - ur[:, fl]) / np.linalg.norm(ur[:, fl]) < 1e-6
    assert np.abs(out[0, fl] - refo[0, fl]).max() < 1e-7
    if solid is not None:
        assert np.array_equal(out[:, ~fl], ref[:, ~fl])
