"""FP64 CPU oracle for the DiffWind hot path (MLS-MPM substep, wind-force
sample, D3Q19 BGK LBM step, the moment-encoded HOME-LBM step, obstacle
voxelization, the learned LBM surrogate) and their adjoints.

TEST INFRASTRUCTURE ONLY. The oracle is the plain, slow, obviously correct
restatement of the method that the CUDA path is checked against. Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import it. It shares no code with the CUDA library and never
imports the product package.

The arithmetic lives in plain C (``mpm_oracle.c``, ``lbm_oracle.c``,
``home_oracle.c``, ``surrogate_oracle.c``), compiled
with gcc into ``_build/liboracle.so``; this module only builds, loads and
marshals numpy float64 arrays. Every function takes and returns
structure-of-arrays data in the layouts the C files document.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = [os.path.join(_HERE, "mpm_oracle.c"), os.path.join(_HERE, "lbm_oracle.c"),
            os.path.join(_HERE, "home_oracle.c"), os.path.join(_HERE, "surrogate_oracle.c")]
_lock = threading.Lock()
_lib = None

ORC_OK = 0
STATUS_NAMES = {0: "ok", 1: "bad argument", 3: "out of memory", 4: "non-finite value",
                5: "particle outside the grid stencil range", 7: "inverted element (det F <= 0)"}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, serial)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SOURCES)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off", "-shared",
               "-fPIC", "-o", tmp] + _SOURCES + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _declare(ct.CDLL(_LIB_PATH))
    return _lib


_dp = ct.POINTER(ct.c_double)
_u8p = ct.POINTER(ct.c_uint8)
_ip = ct.POINTER(ct.c_int)


class _MpmParams(ct.Structure):
    _fields_ = [("n_grid", ct.c_int), ("dt", ct.c_double), ("gravity", ct.c_double * 3),
                ("bc_band", ct.c_int), ("material", ct.c_int), ("E", ct.c_double),
                ("nu", ct.c_double), ("p_mass", ct.c_double), ("p_vol", ct.c_double)]


class _Wind(ct.Structure):
    _fields_ = [("values", _dp), ("nf", ct.c_int), ("n_frames", ct.c_int), ("t_total", ct.c_double)]


def _declare(lib):
    i64 = ct.c_int64
    d = ct.c_double
    i = ct.c_int
    P = ct.POINTER(_MpmParams)
    sig = {
        "orc_lame": (None, [d, d, _dp, _dp]),
        "orc_polar": (i, [_dp, _dp, _dp]),
        "orc_neohookean_psi": (d, [_dp, d, d]),
        "orc_fixedcorot_psi": (d, [_dp, d, d]),
        "orc_stress": (i, [i, _dp, d, d, _dp]),
        "orc_stress_adjoint": (i, [i, _dp, d, d, _dp, _dp]),
        "orc_bspline_weights": (None, [d, _dp]),
        "orc_wind_sample": (None, [_dp, i, i, d, _dp, i64, d, _dp]),
        "orc_wind_sample_adjoint": (None, [_dp, i, i, d, _dp, i64, d, _dp, _dp]),
        "orc_mpm_p2g_grid": (i, [P, i64, _dp, _dp, _dp, _dp, _dp, _dp]),
        "orc_mpm_grid_update": (i, [P, _dp, _dp, ct.POINTER(_Wind), d, _dp]),
        "orc_mpm_g2p": (i, [P, i64, _dp, _dp, _u8p, _dp, _dp, _dp, _dp, _dp]),
        "orc_mpm_substep": (i, [P, i64, _dp, _dp, _dp, _dp, _u8p, _dp, i, i, d, d,
                                _dp, _dp, _dp, _dp]),
        "orc_mpm_substep_adjoint": (i, [P, i64, _dp, _dp, _dp, _dp, _u8p, _dp, i, i, d, d,
                                        _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]),
        "orc_lbm_velocity_set": (None, [_ip, _dp, _ip]),
        "orc_lbm_equilibrium": (None, [d, _dp, _dp]),
        "orc_lbm_collide": (None, [_dp, d, _dp, _dp]),
        "orc_lbm_collide_adjoint": (None, [_dp, d, _dp, _dp, _dp]),
        "orc_lbm_step": (i, [i, i, i, d, _dp, _dp, i, _u8p, _dp, i]),
        "orc_lbm_step_adjoint": (i, [i, i, i, d, _dp, _dp, i, _u8p, _dp, _dp, i]),
        "orc_lbm_macroscopic": (None, [i, i, i, _dp, _u8p, _dp, _dp, _dp]),
        "orc_voxelize": (None, [_dp, i64, i, i, i, d, _u8p]),
        "orc_home_reconstruct": (None, [_dp, _dp]),
        "orc_home_collide": (None, [_dp, d, _dp, _dp]),
        "orc_home_init": (None, [i64, d, _dp, d, _dp, _dp]),
        "orc_home_step": (i, [i, i, i, d, _dp, _dp, i, _u8p, _dp, i]),
        "orc_home_macroscopic": (None, [i64, _dp, _u8p, _dp, _dp, _dp]),
        "orc_surr_num_params": (i64, []),
        "orc_surr_forward": (None, [i, _dp, _dp, _dp, _dp, _dp]),
        "orc_surr_backward": (None, [i, _dp, _dp, _dp, _dp]),
        "orc_surr_features": (None, [i, _dp, _u8p, _dp, _dp, _dp, _dp]),
        "orc_surr_apply": (None, [i, _dp, _dp, _dp, _u8p, _dp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _u8ptr(a):
    return None if a is None else a.ctypes.data_as(_u8p)


def _check(st, what):
    if st != ORC_OK:
        raise OracleError(f"oracle {what}: {STATUS_NAMES.get(st, st)}")


# ------------------------------------------------------------ constitutive --

def lame(E, nu):
    mu, lam = ct.c_double(), ct.c_double()
    _load().orc_lame(E, nu, ct.byref(mu), ct.byref(lam))
    return mu.value, lam.value


def polar(F):
    F = _f64(F, (9,))
    R, S = np.zeros(9), np.zeros(9)
    _check(_load().orc_polar(_ptr(F), _ptr(R), _ptr(S)), "polar")
    return R.reshape(3, 3), S.reshape(3, 3)


def psi(material, F, E, nu):
    mu, lam = lame(E, nu)
    F = _f64(F, (9,))
    fn = _load().orc_neohookean_psi if material == 0 else _load().orc_fixedcorot_psi
    return fn(_ptr(F), mu, lam)


def stress(material, F, E, nu):
    mu, lam = lame(E, nu)
    F = _f64(F, (9,))
    P = np.zeros(9)
    _check(_load().orc_stress(material, _ptr(F), mu, lam, _ptr(P)), "stress")
    return P.reshape(3, 3)


def stress_adjoint(material, F, E, nu, Pbar):
    mu, lam = lame(E, nu)
    F = _f64(F, (9,))
    Pbar = _f64(Pbar, (9,))
    Fbar = np.zeros(9)
    _check(_load().orc_stress_adjoint(material, _ptr(F), mu, lam, _ptr(Pbar), _ptr(Fbar)),
           "stress adjoint")
    return Fbar.reshape(3, 3)


def bspline_weights(fx):
    w = np.zeros(3)
    _load().orc_bspline_weights(float(fx), _ptr(w))
    return w


# -------------------------------------------------------------------- wind --

def wind_sample(values, nf, n_frames, t_total, pos, t):
    """a_w at positions pos[3][n] and time t; returns [3][n]."""
    values = _f64(values)
    pos = _f64(pos)
    n = pos.shape[1]
    out = np.zeros((3, n))
    _load().orc_wind_sample(_ptr(values), nf, n_frames, t_total, _ptr(pos), n, t, _ptr(out))
    return out


def wind_sample_adjoint(values, nf, n_frames, t_total, pos, t, g_out, g_values=None):
    values = _f64(values)
    pos = _f64(pos)
    g_out = _f64(g_out)
    n = pos.shape[1]
    gv = np.zeros(values.shape) if g_values is None else g_values
    _load().orc_wind_sample_adjoint(_ptr(values), nf, n_frames, t_total, _ptr(pos), n, t,
                                    _ptr(g_out), _ptr(gv))
    return gv


# --------------------------------------------------------------------- MPM --

def _params(p):
    return _MpmParams(int(p["n_grid"]), float(p["dt"]), (ct.c_double * 3)(*p["gravity"]),
                      int(p["bc_band"]), int(p["material"]), float(p["E"]), float(p["nu"]),
                      float(p["p_mass"]), float(p["p_vol"]))


def _pinned(pinned, n):
    if pinned is None:
        return None
    return np.ascontiguousarray(np.asarray(pinned, dtype=np.uint8).reshape(n))


def mpm_p2g(params, x, v, C, F):
    """Grid mass m[N^3] and momentum p[3][N^3] after P2G (node index (k*N+j)*N+i)."""
    x, v, C, F = _f64(x), _f64(v), _f64(C), _f64(F)
    n = x.shape[1]
    N = int(params["n_grid"])
    gm = np.zeros(N ** 3)
    gp = np.zeros((3, N ** 3))
    pr = _params(params)
    _check(_load().orc_mpm_p2g_grid(ct.byref(pr), n, _ptr(x), _ptr(v), _ptr(C), _ptr(F),
                                    _ptr(gm), _ptr(gp)), "p2g")
    return gm, gp


def mpm_grid_update(params, gm, gp, wind, t):
    """Grid velocities v[3][N^3] from mass and momentum (Eq. grid update: the
    momentum over the mass plus dt (gravity + wind force), zero on empty
    nodes and in the sticky wall band)."""
    gm, gp = _f64(gm), _f64(gp)
    N = int(params["n_grid"])
    values, nf, nfr, ttot = wind
    values = _f64(values)
    w = _Wind(_ptr(values), int(nf), int(nfr), float(ttot))
    gv = np.zeros((3, N ** 3))
    pr = _params(params)
    _check(_load().orc_mpm_grid_update(ct.byref(pr), _ptr(gm), _ptr(gp), ct.byref(w), float(t),
                                       _ptr(gv)), "grid update")
    return gv


def mpm_g2p(params, x, F, gv, pinned=None):
    """G2P and the deformation update of particles at x with gradients F from
    grid velocities gv[3][N^3]. Returns (x, v, C, F) after the substep."""
    x, F, gv = _f64(x), _f64(F), _f64(gv)
    n = x.shape[1]
    out = (np.zeros((3, n)), np.zeros((3, n)), np.zeros((9, n)), np.zeros((9, n)))
    pr = _params(params)
    pin = _pinned(pinned, n)
    _check(_load().orc_mpm_g2p(ct.byref(pr), n, _ptr(x), _ptr(F), _u8ptr(pin), _ptr(gv),
                               *(_ptr(o) for o in out)), "g2p")
    return out


def mpm_substep(params, state, wind, t, pinned=None):
    """One substep. state = (x[3][n], v[3][n], C[9][n], F[9][n]); wind =
    (values, nf, n_frames, t_total). Returns the new state tuple."""
    x, v, C, F = (_f64(a) for a in state)
    n = x.shape[1]
    values, nf, nfr, ttot = wind
    values = _f64(values)
    out = tuple(np.zeros_like(a) for a in (x, v, C, F))
    pr = _params(params)
    pin = _pinned(pinned, n)
    st = _load().orc_mpm_substep(ct.byref(pr), n, _ptr(x), _ptr(v), _ptr(C), _ptr(F),
                                 _u8ptr(pin), _ptr(values), nf, nfr, ttot, t,
                                 *(_ptr(o) for o in out))
    _check(st, "substep")
    return out


def mpm_substep_adjoint(params, state, wind, t, g_out, pinned=None, g_wind=None):
    """Reverse mode of one substep. Returns (g_state_in, g_wind, g_E) where
    g_wind and g_E accumulate on top of the given g_wind (if any)."""
    x, v, C, F = (_f64(a) for a in state)
    n = x.shape[1]
    values, nf, nfr, ttot = wind
    values = _f64(values)
    go = tuple(_f64(a) for a in g_out)
    gi = tuple(np.zeros_like(a) for a in (x, v, C, F))
    gw = np.zeros(values.shape) if g_wind is None else g_wind
    gE = ct.c_double(0.0)
    pr = _params(params)
    pin = _pinned(pinned, n)
    st = _load().orc_mpm_substep_adjoint(ct.byref(pr), n, _ptr(x), _ptr(v), _ptr(C), _ptr(F),
                                         _u8ptr(pin), _ptr(values), nf, nfr, ttot, t,
                                         *(_ptr(a) for a in go), *(_ptr(a) for a in gi),
                                         _ptr(gw), ct.byref(gE))
    _check(st, "substep adjoint")
    return gi, gw, gE.value


def mpm_rollout(params, state, wind, t0, n_substeps, pinned=None, keep_every=0):
    """n_substeps substeps from time t0; optionally also returns the states at
    every keep_every-th substep boundary (including the initial state)."""
    dt = float(params["dt"])
    kept = []
    s = tuple(_f64(a) for a in state)
    for k in range(n_substeps):
        if keep_every and k % keep_every == 0:
            kept.append(s)
        s = mpm_substep(params, s, wind, t0 + k * dt, pinned)
    if keep_every:
        kept.append(s)
        return s, kept
    return s


# --------------------------------------------------------------------- LBM --

def velocity_set():
    c = np.zeros((19, 3), dtype=np.intc)
    w = np.zeros(19)
    op = np.zeros(19, dtype=np.intc)
    _load().orc_lbm_velocity_set(c.ctypes.data_as(_ip), _ptr(w), op.ctypes.data_as(_ip))
    return c, w, op


def lbm_equilibrium(rho, u):
    u = _f64(u, (3,))
    feq = np.zeros(19)
    _load().orc_lbm_equilibrium(float(rho), _ptr(u), _ptr(feq))
    return feq


def lbm_collide(f, tau, force=(0.0, 0.0, 0.0)):
    f = _f64(f, (19,))
    force = _f64(force, (3,))
    out = np.zeros(19)
    _load().orc_lbm_collide(_ptr(f), tau, _ptr(force), _ptr(out))
    return out


def lbm_collide_adjoint(f, tau, gpost, force=(0.0, 0.0, 0.0)):
    f = _f64(f, (19,))
    force = _f64(force, (3,))
    gpost = _f64(gpost, (19,))
    out = np.zeros(19)
    _load().orc_lbm_collide_adjoint(_ptr(f), tau, _ptr(force), _ptr(gpost), _ptr(out))
    return out


def _mask(solid, nc):
    if solid is None:
        return None
    return np.ascontiguousarray(np.asarray(solid, dtype=np.uint8).reshape(nc))


def lbm_step(shape, tau, f, steps, u_in=(0.0, 0.0, 0.0), force=(0.0, 0.0, 0.0), bc_x=0,
             solid=None):
    """Advance populations f[19][nz*ny*nx] (plain, unshifted) by `steps`."""
    nx, ny, nz = shape
    f = _f64(f).copy()
    u_in = _f64(u_in, (3,))
    force = _f64(force, (3,))
    m = _mask(solid, nx * ny * nz)
    st = _load().orc_lbm_step(nx, ny, nz, tau, _ptr(u_in), _ptr(force), bc_x, _u8ptr(m),
                              _ptr(f), steps)
    _check(st, "lbm step")
    return f


def lbm_step_adjoint(shape, tau, f0, g, steps, u_in=(0.0, 0.0, 0.0), force=(0.0, 0.0, 0.0),
                     bc_x=0, solid=None):
    nx, ny, nz = shape
    f0 = _f64(f0)
    g = _f64(g).copy()
    u_in = _f64(u_in, (3,))
    force = _f64(force, (3,))
    m = _mask(solid, nx * ny * nz)
    st = _load().orc_lbm_step_adjoint(nx, ny, nz, tau, _ptr(u_in), _ptr(force), bc_x,
                                      _u8ptr(m), _ptr(f0), _ptr(g), steps)
    _check(st, "lbm step adjoint")
    return g


def lbm_macroscopic(shape, f, force=(0.0, 0.0, 0.0), solid=None):
    nx, ny, nz = shape
    nc = nx * ny * nz
    f = _f64(f)
    force = _f64(force, (3,))
    rho = np.zeros(nc)
    u = np.zeros((3, nc))
    m = _mask(solid, nc)
    _load().orc_lbm_macroscopic(nx, ny, nz, _ptr(force), _u8ptr(m), _ptr(f), _ptr(rho), _ptr(u))
    return rho, u


# ---------------------------------------------------------------- HOME-LBM --

def home_reconstruct(m):
    """The 19 populations of one cell's moments m[10] (rho, u, Sxx, Syy, Szz,
    Sxy, Sxz, Syz)."""
    m = _f64(m, (10,))
    f = np.zeros(19)
    _load().orc_home_reconstruct(_ptr(m), _ptr(f))
    return f


def home_collide(f, tau, force=(0.0, 0.0, 0.0)):
    """The stored moments m[10] after the moment-space collision of one
    cell's pre-collision populations f[19]."""
    f = _f64(f, (19,))
    force = _f64(force, (3,))
    m = np.zeros(10)
    _load().orc_home_collide(_ptr(f), float(tau), _ptr(force), _ptr(m))
    return m


def home_init(shape, rho0, u0, tau, force=(0.0, 0.0, 0.0)):
    """m[10][nz*ny*nx]: every cell the collided equilibrium f_eq(rho0, u0)."""
    nx, ny, nz = shape
    nc = nx * ny * nz
    u0 = _f64(u0, (3,))
    force = _f64(force, (3,))
    m = np.zeros((10, nc))
    _load().orc_home_init(nc, float(rho0), _ptr(u0), float(tau), _ptr(force), _ptr(m))
    return m


def home_step(shape, tau, m, steps, u_in=(0.0, 0.0, 0.0), force=(0.0, 0.0, 0.0), bc_x=0,
              solid=None):
    """Advance moments m[10][nz*ny*nx] by `steps` HOME-LBM steps."""
    nx, ny, nz = shape
    m = _f64(m).copy()
    u_in = _f64(u_in, (3,))
    force = _f64(force, (3,))
    mask = _mask(solid, nx * ny * nz)
    st = _load().orc_home_step(nx, ny, nz, float(tau), _ptr(u_in), _ptr(force), bc_x,
                               _u8ptr(mask), _ptr(m), steps)
    _check(st, "home step")
    return m


def home_macroscopic(shape, m, force=(0.0, 0.0, 0.0), solid=None):
    nx, ny, nz = shape
    nc = nx * ny * nz
    m = _f64(m)
    force = _f64(force, (3,))
    rho = np.zeros(nc)
    u = np.zeros((3, nc))
    mask = _mask(solid, nc)
    _load().orc_home_macroscopic(nc, _ptr(force), _u8ptr(mask), _ptr(m), _ptr(rho), _ptr(u))
    return rho, u


def voxelize(pos, shape, dx):
    """Eq. point2voxel mask uint8[nz*ny*nx] from particle positions pos[3][n]."""
    nx, ny, nz = shape
    pos = _f64(pos)
    solid = np.zeros(nx * ny * nz, dtype=np.uint8)
    _load().orc_voxelize(_ptr(pos), pos.shape[1], nx, ny, nz, float(dx), _u8ptr(solid))
    return solid


# --------------------------------------------------------------- surrogate --

SURR_CHANNELS = (16, 32, 32, 32, 16)


def surr_num_params():
    return int(_load().orc_surr_num_params())


def surr_layer_slices():
    """[(W slice, b slice, cin, cout)] into the packed parameter vector; W is
    [27][cout][cin], tap = (dz+1)*9 + (dy+1)*3 + (dx+1)."""
    out, o = [], 0
    for l in range(4):
        cin, cout = SURR_CHANNELS[l], SURR_CHANNELS[l + 1]
        nw = 27 * cin * cout
        out.append((slice(o, o + nw), slice(o + nw, o + nw + cout), cin, cout))
        o += nw + cout
    return out


def surr_forward(n, params, feats, keep=False):
    """feats [n^3][16] channels-last -> out [n^3][16] (and the hidden z, a)."""
    params = _f64(params)
    feats = _f64(feats)
    nv = n ** 3
    out = np.zeros((nv, 16))
    z = np.zeros((3, nv, 32)) if keep else None
    a = np.zeros((3, nv, 32)) if keep else None
    _load().orc_surr_forward(n, _ptr(params), _ptr(feats), _ptr(z), _ptr(a), _ptr(out))
    return (out, z, a) if keep else out


def surr_backward(n, params, feats, g_out):
    params = _f64(params)
    feats = _f64(feats)
    g_out = _f64(g_out)
    g = np.zeros_like(params)
    _load().orc_surr_backward(n, _ptr(params), _ptr(feats), _ptr(g_out), _ptr(g))
    return g


def surr_features(n, f, solid=None, u_ref=(0.0, 0.0, 0.0)):
    """Coarse features [n^3][16] of a fine (2n)^3 lattice of plain populations
    f[19][cells] (velocities relative to u_ref, u_ref itself in channels 5-7),
    with the fine rho [cells] and u [3][cells]."""
    f = _f64(f)
    N3 = (2 * n) ** 3
    feats = np.zeros((n ** 3, 16))
    rho = np.zeros(N3)
    u = np.zeros((3, N3))
    m = _mask(solid, N3)
    ur = np.ascontiguousarray(np.asarray(u_ref, np.float64))
    _load().orc_surr_features(n, _ptr(f), _u8ptr(m), _ptr(ur), _ptr(feats), _ptr(rho), _ptr(u))
    return feats, rho, u


def surr_apply(n, du, rho_fine, u_fine, f, solid=None):
    """f (plain, [19][cells]) re-initialised to f_eq(rho, u + upsampled du)."""
    du = _f64(du)
    rho_fine = _f64(rho_fine)
    u_fine = _f64(u_fine)
    f = _f64(f).copy()
    m = _mask(solid, (2 * n) ** 3)
    _load().orc_surr_apply(n, _ptr(du), _ptr(rho_fine), _ptr(u_fine), _u8ptr(m), _ptr(f))
    return f
