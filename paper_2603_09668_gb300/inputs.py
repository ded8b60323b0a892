"""Seeded synthetic inputs shaped like DiffWind's wind-driven scenes.

This module holds input generation only: particle clouds, random wind-force
keyframes, obstacle clusters and random perturbations. It contains none of the
method's arithmetic (no weights, transfers, stresses, equilibria or voxel
rules), so both the CUDA path and the CPU oracle can be fed from it.

The paper's scenes come from its WD-Objects captures, which are not available;
these generators stand in for them with the shapes the paper describes:
leaves, flags and fabrics (thin sheets pinned along one edge), solid blocks,
and a cluster of leaf-like ellipsoidal patches as the LBM obstacle. Grid sizes
(128^3, Sec. 4.1), particle counts (52k-146k object particles per scene,
Table sim_time) and Young's moduli (4e4 / 4e5 / 4e6, Table ablation_physical)
follow the paper's scale.

Every generator is a pure function of its arguments and seed
(numpy PCG64 streams) and returns float32 numpy arrays in the
structure-of-arrays layout of the C-ABI: positions [3][n], C and F [9][n].
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ------------------------------------------------------------- particles --

def block_particles(lo=(0.375, 0.275, 0.375), size=0.25, sub=16, per_sub=2, seed=0):
    """Jittered stratified samples in a cube: a sub^3 lattice of sub-cells with
    per_sub uniform samples each (sub=16, per_sub=2 gives 8192 particles)."""
    g = rng(seed)
    h = size / sub
    idx = np.stack(np.meshgrid(np.arange(sub), np.arange(sub), np.arange(sub), indexing="ij"),
                   axis=-1).reshape(-1, 3)
    idx = np.repeat(idx, per_sub, axis=0)
    pts = (idx + g.random(idx.shape)) * h + np.asarray(lo)
    return np.ascontiguousarray(pts.T.astype(np.float32))


def sheet_particles(nu=548, nv=365, layers=2, x_range=(0.2, 0.8), y_range=(0.4, 0.8), z0=0.5,
                    jitter=0.0, seed=0):
    """A flag-like thin sheet in the x-y plane: an nu x nv lattice of particles
    per layer, `layers` layers one lattice spacing apart in z, centred on z0.
    Returns (positions [3][n], pinned uint8[n]) where the pinned particles are
    the column with the smallest x (the flag's edge on its pole)."""
    g = rng(seed)
    xs = np.linspace(x_range[0], x_range[1], nu)
    ys = np.linspace(y_range[0], y_range[1], nv)
    h = xs[1] - xs[0]
    zs = z0 + (np.arange(layers) - 0.5 * (layers - 1)) * h
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=0)
    if jitter > 0.0:
        pts = pts + (g.random(pts.shape) - 0.5) * jitter * h
    pinned = np.zeros(pts.shape[1], dtype=np.uint8)
    pinned[np.isclose(X.ravel(), xs[0])] = 1
    return np.ascontiguousarray(pts.astype(np.float32)), pinned


def ellipsoid_cluster(n_patches=50, per_patch=4000, r_lo=0.02, r_hi=0.06, c_lo=0.3, c_hi=0.7,
                      seed=0):
    """Leaf cluster: n_patches ellipsoids with semi-axes U[r_lo, r_hi], random
    orientation and centres U[c_lo, c_hi]^3, each filled with per_patch
    uniformly distributed particles. Returns positions [3][n]."""
    g = rng(seed)
    out = []
    for _ in range(n_patches):
        axes = g.uniform(r_lo, r_hi, size=3)
        centre = g.uniform(c_lo, c_hi, size=3)
        q, r = np.linalg.qr(g.standard_normal((3, 3)))
        q = q * np.sign(np.diag(r))
        d = g.standard_normal((per_patch, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        rad = g.random(per_patch) ** (1.0 / 3.0)
        local = d * rad[:, None] * axes[None, :]
        out.append(local @ q.T + centre[None, :])
    pts = np.concatenate(out, axis=0).T
    return np.ascontiguousarray(pts.astype(np.float32))


def rest_state(x):
    """v = 0, C = 0, F = I for positions x[3][n]."""
    n = x.shape[1]
    v = np.zeros((3, n), np.float32)
    C = np.zeros((9, n), np.float32)
    F = np.zeros((9, n), np.float32)
    F[[0, 4, 8]] = 1.0
    return np.ascontiguousarray(x.astype(np.float32)), v, C, F


def perturbed_state(x, v_scale=0.1, c_scale=1.0, f_scale=0.02, seed=1):
    """A random non-rest state: uniform velocities in [-v_scale, v_scale],
    affine matrices in [-c_scale, c_scale] and F = I + U[-f_scale, f_scale]."""
    g = rng(seed)
    n = x.shape[1]
    v = (g.uniform(-v_scale, v_scale, (3, n))).astype(np.float32)
    C = (g.uniform(-c_scale, c_scale, (9, n))).astype(np.float32)
    F = (g.uniform(-f_scale, f_scale, (9, n))).astype(np.float32)
    F[[0, 4, 8]] += 1.0
    return np.ascontiguousarray(x.astype(np.float32)), v, C, F


# ------------------------------------------------------------------ wind --

def constant_wind(nf, n_frames, vec):
    vals = np.empty((n_frames, nf, nf, nf, 3), np.float32)
    vals[...] = np.asarray(vec, np.float32)
    return vals


def fourier_wind(nf, n_frames, mean=(10.0, 0.0, 0.0), amp=2.0, n_modes=8, kmax=3, seed=0):
    """Smooth random wind-force keyframes [n_frames][nf][nf][nf][3] (x fastest
    in the spatial index): per component, mean + sum of n_modes cosines
    amp * cos(2 pi (k . x + w s) + phi) with integer wave vectors k in
    {-kmax..kmax}^3 minus 0, w ~ U[0, 2] cycles over the keyframe span
    (s = frame / (n_frames - 1)) and phi ~ U[0, 2 pi). With amp = 2 and 8 modes
    the standard deviation is sqrt(8 amp^2 / 2) = 4."""
    g = rng(seed)
    grid = np.linspace(0.0, 1.0, nf) if nf > 1 else np.zeros(1)
    Z, Y, X = np.meshgrid(grid, grid, grid, indexing="ij")
    s = np.linspace(0.0, 1.0, n_frames) if n_frames > 1 else np.zeros(1)
    vals = np.zeros((n_frames, nf, nf, nf, 3), np.float64)
    for c in range(3):
        vals[..., c] = mean[c]
        for _ in range(n_modes):
            while True:
                k = g.integers(-kmax, kmax + 1, size=3)
                if np.any(k != 0):
                    break
            w = g.uniform(0.0, 2.0)
            phi = g.uniform(0.0, 2.0 * np.pi)
            spatial = k[0] * X + k[1] * Y + k[2] * Z
            for f in range(n_frames):
                vals[f, ..., c] += amp * np.cos(2.0 * np.pi * (spatial + w * s[f]) + phi)
    return np.ascontiguousarray(vals.astype(np.float32))


def wind_node_positions(nf):
    """Positions [3][nf^3] (float32, x index fastest) of the wind-grid nodes,
    node (i, j, k) at (i, j, k) / (nf - 1): the node-centred grid spanning the
    unit cube on which the wind keyframes are stored."""
    grid = np.linspace(0.0, 1.0, nf) if nf > 1 else np.zeros(1)
    Z, Y, X = np.meshgrid(grid, grid, grid, indexing="ij")
    return np.ascontiguousarray(np.stack([X.ravel(), Y.ravel(), Z.ravel()]).astype(np.float32))


# ------------------------------------------------------------------- LBM --

def population_noise(shape, amplitude=1e-3, seed=0):
    """Uniform noise [19][nz*ny*nx] in [-amplitude, amplitude], used to start
    lattices away from rest."""
    nx, ny, nz = shape
    return rng(seed).uniform(-amplitude, amplitude, (19, nx * ny * nz)).astype(np.float32)


def random_mask(shape, fraction=0.05, seed=0):
    nx, ny, nz = shape
    return (rng(seed).random(nx * ny * nz) < fraction).astype(np.uint8)


# ---------------------------------------------------------------- scenes --

@dataclass
class Scene:
    """One MPM scene: grid, material, time step, particles and wind."""
    name: str
    n_grid: int
    dt: float
    material: int  # 0 Neo-Hookean, 1 fixed-corotated
    E: float
    nu: float
    rho: float
    p_vol: float
    x: np.ndarray
    pinned: np.ndarray | None
    wind: np.ndarray  # [n_frames][nf][nf][nf][3]
    t_total: float
    gravity: tuple = (0.0, -9.8, 0.0)
    bc_band: int = 3
    n_substeps: int = 100
    extra: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.x.shape[1]

    @property
    def p_mass(self):
        return self.rho * self.p_vol

    @property
    def nf(self):
        return self.wind.shape[1]

    @property
    def n_frames(self):
        return self.wind.shape[0]

    def params(self):
        return dict(n_grid=self.n_grid, dt=self.dt, gravity=self.gravity, bc_band=self.bc_band,
                    material=self.material, E=self.E, nu=self.nu, p_mass=self.p_mass,
                    p_vol=self.p_vol)

    def wind_tuple(self):
        return (self.wind, self.nf, self.n_frames, self.t_total)


def block_scene(seed=0):
    """Forward block: 32^3 grid, 8192 jittered particles in a 0.25 cube centred
    at (0.5, 0.4, 0.5), fixed-corotated E=1e4 nu=0.3 rho=1000, constant 5 N/kg
    wind in +x on an 8^3 grid, dt=1e-4, 100 substeps."""
    x = block_particles(seed=seed)
    return Scene("block32", 32, 1e-4, 1, 1e4, 0.3, 1000.0, 0.25 ** 3 / x.shape[1], x, None,
                 constant_wind(8, 1, (5.0, 0.0, 0.0)), 100 * 1e-4, n_substeps=100)


def sheet_scene(nu=548, nv=365, n_grid=128, n_substeps=1000, dt=5e-5, wind_nf=32, wind_frames=16,
                seed=0, wind_seed=0, E=5e4):
    """Flag-like sheet: 0.6 x 0.4 sheet, 2 particles thick, pinned along its
    x = 0.2 edge, Neo-Hookean E=5e4 nu=0.3 rho=1000, Fourier wind (mean 10 N/kg
    +x, std 4) on a wind_nf^3 x wind_frames grid over the rollout, dt=5e-5."""
    x, pinned = sheet_particles(nu, nv, seed=seed)
    h = 0.6 / (nu - 1)
    vol = 0.6 * 0.4 * 2 * h
    t_total = n_substeps * dt
    wind = fourier_wind(wind_nf, wind_frames, seed=wind_seed)
    return Scene(f"sheet{n_grid}", n_grid, dt, 0, E, 0.3, 1000.0, vol / x.shape[1], x, pinned,
                 wind, t_total, n_substeps=n_substeps)


def sheet_texture(x, cell=0.05):
    """Colours [3][n] of a checkerboard of `cell`-sized squares over the rest
    positions x [3][n] (x-y plane): 0.85 / 0.2 per square, a different tint
    per channel."""
    sq = (np.floor(x[0] / cell) + np.floor(x[1] / cell)).astype(np.int64) % 2
    base = np.where(sq == 1, 0.85, 0.2)
    tint = np.array([1.0, 0.8, 0.6])[:, None]
    return np.ascontiguousarray((tint * base[None, :]).astype(np.float32))


def inversion_case(nu=64, nv=43, n_grid=64, nf=12, n_intervals=3, substeps=200, dt=2e-4,
                   every=25, n_cells=32, lbm_steps=30, inlet_error_deg=10.0, lbm_model="home",
                   seed=0):
    """Synthetic wind-inversion case: the flag-like sheet (pinned edge, E=5e4)
    on an n_grid^3 grid, n_intervals intervals of `substeps` substeps of dt
    (0.04 s, a video frame interval; checkpoint every `every`), a wind grid of
    nf^3 nodes, and an n_cells^3 lattice (tau 0.6; HOME-LBM, or BGK with
    lbm_model="bgk") with an inlet of speed 0.05 along (1, 0, 0.35) advanced
    lbm_steps steps per interval. The ground-truth
    force follows the drag relation with scale 4000 (10 N/kg at the inlet
    speed); the inversion's guide lattice assumes a wind-source direction off
    by inlet_error_deg degrees about y."""
    sc = sheet_scene(nu, nv, n_grid=n_grid, n_substeps=substeps, dt=dt, wind_nf=nf,
                     wind_frames=1, seed=seed)
    d = np.array([1.0, 0.0, 0.35])
    u_in = tuple(float(c) for c in 0.05 * d / np.linalg.norm(d))
    return dict(scene=sc, nu=nu, nf=nf, n_intervals=n_intervals, substeps=substeps, every=every,
                n_cells=n_cells, tau=0.6, u_inlet=u_in, drag_scale=4000.0, lbm_steps=lbm_steps,
                inlet_error_deg=inlet_error_deg, lbm_model=lbm_model)


def gaussian_scene(n=300, width=61, height=47, depth_ties=False, seed=0):
    """Particle-bound Gaussians for the renderer: centres uniform in a 0.8
    box, deformation gradients I + U[-0.15, 0.15] per entry, rest covariances
    with standard deviations in [0.01, 0.04] along random axes, colours U[0, 1],
    opacities U[0.2, 0.95]. The camera looks at the box from 2.2 units,
    rotated 0.3 rad about (0.2, 1, 0.1), focal length 0.9 width. With
    depth_ties the camera is not rotated and every fourth Gaussian copies the
    z of its predecessor, so that the depth keys tie exactly in any precision
    (the order is then the index order). Returns (x, F, sigma0, color,
    opacity, camera dict), arrays float32."""
    g = rng(seed)
    x = g.uniform(-0.4, 0.4, (3, n))
    F = g.uniform(-0.15, 0.15, (9, n))
    F[[0, 4, 8]] += 1.0
    sig = np.zeros((6, n))
    for p in range(n):
        q, _ = np.linalg.qr(g.standard_normal((3, 3)))
        S = q @ np.diag(g.uniform(0.01, 0.04, 3) ** 2) @ q.T
        sig[:, p] = [S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]]
    if depth_ties:
        R = np.eye(3)
        x[2, 4::4] = x[2, 3:-1:4][: len(x[2, 4::4])]
    else:
        a = np.array([0.2, 1.0, 0.1]) / np.linalg.norm([0.2, 1.0, 0.1])
        K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
        R = np.eye(3) + np.sin(0.3) * K + (1 - np.cos(0.3)) * K @ K
    T = np.array([0.0, 0.0, 2.2])
    color = g.uniform(0.0, 1.0, (3, n))
    opacity = g.uniform(0.2, 0.95, n)
    cam = dict(R=R, T=T, fx=0.9 * width, fy=0.9 * width, cx=width / 2, cy=height / 2,
               width=width, height=height)
    f32 = lambda a: np.ascontiguousarray(a.astype(np.float32))
    return f32(x), f32(F), f32(sig), f32(color), f32(opacity), cam


def batch_scenes(n_scenes=64, n_lo=20000, n_hi=400000, n_substeps=500, seed=0):
    """Uneven multi-scene batch: particle counts log-uniform in [n_lo, n_hi],
    grid 64^3 or 128^3, sheet or block, each with its own 16^3 x 8 wind."""
    g = rng(seed)
    scenes = []
    for s in range(n_scenes):
        n_target = int(np.exp(g.uniform(np.log(n_lo), np.log(n_hi))))
        n_grid = 64 if g.random() < 0.5 else 128
        sheet = g.random() < 0.5
        dt = 5e-5
        wind = fourier_wind(16, 8, seed=1000 + s)
        if sheet:
            # aspect 3:2 lattice, 2 layers
            nv = max(8, int(np.sqrt(n_target / 2 / 1.5)))
            nu = max(8, int(n_target / 2 / nv))
            x, pinned = sheet_particles(nu, nv, seed=s)
            h = 0.6 / (nu - 1)
            vol = 0.6 * 0.4 * 2 * h
            scenes.append(Scene(f"b{s}_sheet{n_grid}", n_grid, dt, 0, 5e4, 0.3, 1000.0,
                                vol / x.shape[1], x, pinned, wind, n_substeps * dt,
                                n_substeps=n_substeps))
        else:
            sub = max(4, int(round((n_target / 2) ** (1.0 / 3.0))))
            x = block_particles(sub=sub, seed=s)
            scenes.append(Scene(f"b{s}_block{n_grid}", n_grid, dt, 1, 1e4, 0.3, 1000.0,
                                0.25 ** 3 / x.shape[1], x, None, wind, n_substeps * dt,
                                n_substeps=n_substeps))
    return scenes
