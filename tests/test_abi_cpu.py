"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU,
exports exactly the entry points include/*.h declares, and its ctypes layouts
match the C structs. No compute call is made here."""
import ctypes as ct
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"^DW_API\s+[\w\s\*]*?\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2603_09668_gb300 import build

    return build.build_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mpm_create", "mpm_destroy", "mpm_substep", "mpm_substep_adjoint", "lbm_step",
                     "lbm_step_adjoint", "wind_field_sample", "wind_field_sample_adjoint"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ct.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} is declared in include/ but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert exported == set(declared_functions()), exported ^ set(declared_functions())


def test_ctypes_struct_layouts_match_c(libpath, tmp_path):
    """Compile a tiny C program against the header that prints sizeof/offsetof."""
    from paper_2603_09668_gb300 import _capi

    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "diffwind.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(dw_mpm_desc), offsetof(dw_mpm_desc, max_particles),
         offsetof(dw_mpm_desc, p2g_mode), offsetof(dw_mpm_desc, p_vol));
  printf("%zu %zu\\n", sizeof(dw_mpm_state), offsetof(dw_mpm_state, n));
  printf("%zu %zu\\n", sizeof(dw_wind_field), offsetof(dw_wind_field, t_total));
  printf("%zu %zu %zu\\n", sizeof(dw_lbm_desc), offsetof(dw_lbm_desc, bc_x), offsetof(dw_lbm_desc, max_tape));
  printf("%zu %zu %zu\\n", sizeof(dw_camera), offsetof(dw_camera, width), offsetof(dw_camera, near_z));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    d = _capi.DwMpmDesc
    assert lines[0].split() == [str(ct.sizeof(d)), str(d.max_particles.offset), str(d.p2g_mode.offset),
                                str(d.p_vol.offset)]
    s = _capi.DwMpmState
    assert lines[1].split() == [str(ct.sizeof(s)), str(s.n.offset)]
    w = _capi.DwWindField
    assert lines[2].split() == [str(ct.sizeof(w)), str(w.t_total.offset)]
    lb = _capi.DwLbmDesc
    assert lines[3].split() == [str(ct.sizeof(lb)), str(lb.bc_x.offset), str(lb.max_tape.offset)]
    cm = _capi.DwCamera
    assert lines[4].split() == [str(ct.sizeof(cm)), str(cm.width.offset), str(cm.near_z.offset)]


def test_version_and_error_string_without_gpu(libpath):
    from paper_2603_09668_gb300 import _capi

    L = _capi.lib()
    assert b"sm_103a" in L.dw_version()
    assert L.dw_last_error() == b""


def test_argument_errors_are_reported_without_touching_the_gpu(libpath):
    """Host-side validation runs before any CUDA call, so it works on a CPU machine."""
    from paper_2603_09668_gb300 import _capi

    L = _capi.lib()
    d = _capi.DwMpmDesc(4, 1e-4, (ct.c_float * 3)(0, -9.8, 0), 3, 0, 1e4, 0.3, 1.0, 1.0, 10, 0)
    h = ct.c_void_p()
    assert L.mpm_create(ct.byref(d), ct.byref(h)) == 1  # n_grid < 8
    assert b"n_grid" in L.dw_last_error()
    ld = _capi.DwLbmDesc(32, 32, 32, 0.4, (ct.c_float * 3)(), (ct.c_float * 3)(), 0, 1)
    assert L.lbm_create(ct.byref(ld), ct.byref(h)) == 1  # tau <= 0.5
    assert b"tau" in L.dw_last_error()
    w = _capi.DwWindField(None, 8, 1, 1.0)
    assert L.wind_field_sample(ct.byref(w), None, 0, 0.0, None, None) == 1
    assert L.lbm_step(None, None, None, 2, None) == 1
    assert L.mpm_substep(None, None, None, None, None, 0.0, None) == 1


def test_product_path_fails_loudly_without_the_library(monkeypatch, tmp_path):
    from paper_2603_09668_gb300 import _capi

    monkeypatch.setattr(_capi, "_lib", None)
    monkeypatch.setattr(_capi, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        _capi.lib()


def test_every_declared_entry_point_has_a_ctypes_signature():
    """The Python binding marshals every entry point include/*.h declares."""
    src = open(os.path.join(ROOT, "paper_2603_09668_gb300", "_capi.py")).read()
    missing = [n for n in declared_functions() if f'"{n}"' not in src]
    assert not missing, missing


def _write_state_file(path, n, t, substep, flags, rows=None, extra=b""):
    """A checkpoint in the format include/diffwind.h documents for
    mpm_state_save, written here with numpy (the header reader is host
    code and needs no GPU)."""
    import numpy as np

    with open(path, "wb") as f:
        f.write(b"DWMPMST1")
        f.write(np.array([n], "<i8").tobytes() + np.array([t], "<f8").tobytes())
        f.write(np.array([substep], "<i8").tobytes() + np.array([flags, 0], "<i4").tobytes())
        rows = np.zeros((24, n), "<f4") if rows is None else rows
        f.write(rows.tobytes())
        if flags & 1:
            f.write(np.zeros(n, np.uint8).tobytes())
        if flags & 2:
            f.write(np.arange(n, dtype="<i4").tobytes())
        f.write(extra)


def test_state_checkpoint_header_is_read_without_a_gpu(tmp_path, libpath):
    from paper_2603_09668_gb300 import binding as B

    p = tmp_path / "s.dwst"
    _write_state_file(p, 7, 0.125, 2500, 3)
    assert B.mpm_state_peek(str(p)) == dict(n=7, has_pinned=True, has_ids=True, t=0.125,
                                            substep=2500)
    _write_state_file(p, 5, 1.5, 3, 0)
    h = B.mpm_state_peek(str(p))
    assert (h["n"], h["has_pinned"], h["has_ids"], h["substep"]) == (5, False, False, 3)
    bad = tmp_path / "bad.dwst"
    bad.write_bytes(b"NOTSTATE" + bytes(32))
    with pytest.raises(B.DiffWindError, match="DW_ERR_IO"):
        B.mpm_state_peek(str(bad))
    bad.write_bytes(b"DWMPM")  # short header
    with pytest.raises(B.DiffWindError, match="DW_ERR_IO"):
        B.mpm_state_peek(str(bad))
    with pytest.raises(B.DiffWindError, match="DW_ERR_IO"):
        B.mpm_state_peek(str(tmp_path / "missing.dwst"))


def test_rollout_launch_count_follows_the_launch_sequence():
    """The kernel count the bench reports (`gpu_launches`) for one rollout:
    one P2G, a grid update per substep, a fused launch per substep but the
    last, one G2P, per sort the scan (two kernels up to 1024 scan blocks of
    8192 counters, else three) and the scatter-move, and the key kernel for
    the first sort only when the paired fused kernel counts the later keys."""
    from types import SimpleNamespace

    from paper_2603_09668_gb300 import binding as B
    from paper_2603_09668_gb300.rollout import Rollout

    def count(n_grid, n_sub, sort_every, mode=B.P2G_AUTO):
        mpm = SimpleNamespace(n_grid=n_grid, p2g_mode=mode)
        return Rollout(mpm, 8, None, n_sub, sort_every=sort_every, device="cpu").kernel_launches

    # 128^3: 64 * 32^3 counters = 256 scan blocks; 67 sorts in 1000 substeps
    assert count(128, 1000, 15) == 1 + 2000 + 67 * 3 + 1
    assert count(128, 1000, 0) == 1 + 2000
    assert count(128, 30, 15) == 1 + 60 + 2 * 3 + 1  # sorts at substeps 0 and 15
    # the one-particle fused kernel leaves every sort its key kernel
    assert count(128, 1000, 15, B.P2G_WARP) == 1 + 2000 + 67 * 4
    # 512^3: 64 * 128^3 counters = 16384 scan blocks, a three-kernel scan
    assert count(512, 100, 50) == 1 + 200 + 2 * 4 + 1
