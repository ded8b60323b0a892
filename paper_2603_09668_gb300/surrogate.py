"""Surrogate-accelerated LBM wind constraint.

The plain D3Q19 LBM (lbm_step) advances the wind velocity field one lattice
step at a time. The surrogate advances it by a block of `block` steps in one
network call. The call reads the coarse features of the current lattice,
runs the network, upsamples the predicted change of the coarse velocity,
adds it to the fine velocity and re-initialises the populations at
equilibrium. Training data come from the library's own LBM runs on lattices
with random leaf-cluster obstacles and random inlet directions.

`SurrogateLBM.advance` re-checks the surrogate against the plain LBM every
`check_every` blocks: it runs both from the same lattice and compares the
fluid velocities; the run continues from the plain result. If the relative
L2 error exceeds `tol` (2%), the surrogate is switched off from then on. The
default check interval, 3 blocks, is the one measured to keep a 25-block
run within 2% of the plain LBM's own trajectory on held-out scenes; each
block's error is far smaller (about 0.3%), but chained blocks drift.
"""
from __future__ import annotations

import math
import os

import numpy as np
import torch

from . import binding as B
from . import inputs

U_REF = 0.05        # inlet speed (lattice units)
IN_SCALE = 1.0 / U_REF
OUT_SCALE = 1e-3    # network outputs du / OUT_SCALE
BLOCK = 20          # lattice steps per surrogate call
WEIGHTS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")


def inlet_direction(rng, cone_deg=30.0):
    """Unit vector uniformly distributed in a cone of half-angle cone_deg about +x."""
    cos_max = math.cos(math.radians(cone_deg))
    c = rng.uniform(cos_max, 1.0)
    phi = rng.uniform(0.0, 2.0 * math.pi)
    s = math.sqrt(max(0.0, 1.0 - c * c))
    return np.array([c, s * math.cos(phi), s * math.sin(phi)])


def leaf_mask(N, seed, device="cuda"):
    """Solid mask of the leaf cluster (50 ellipsoids, 200k particles) on N^3."""
    pts = torch.from_numpy(inputs.ellipsoid_cluster(seed=seed)).to(device)
    solid = torch.empty((N, N, N), dtype=torch.uint8, device=device)
    B.voxelize_particles(pts, (N, N, N), 1.0 / N, solid)
    return solid


# channels of the features kept for training (the others are zero)
X_CH = 8
Y_CH = 3


def turned(d, deg, rng):
    """d rotated by `deg` degrees about a random axis normal to it."""
    a = np.cross(d, rng.standard_normal(3))
    a /= np.linalg.norm(a)
    t = math.radians(deg)
    return d * math.cos(t) + np.cross(a, d) * math.sin(t) + a * np.dot(a, d) * (1 - math.cos(t))


def generate_pairs(N, n_rollouts, t_lo, t_hi, seed=0, block=BLOCK, tau=0.55, device="cuda",
                   keep_states=False, per_rollout=1, inlet_features=True, turn_frac=0.0,
                   turn_deg=20.0, turn_window=300):
    """Training pairs from the plain LBM: per rollout a random obstacle and inlet
    direction, a run from rest through `per_rollout` random times in
    [t_lo, t_hi); at each, the coarse features (input, channels 0..X_CH-1) and
    the change of the coarse velocity over the next `block` steps divided by
    OUT_SCALE (target, channels 0..2). A fraction turn_frac of the rollouts turns the inlet
    by turn_deg degrees at a time in [t_lo, t_hi) and samples its pairs in
    the turn_window steps after the turn. Pairs are kept in these compact
    channels (expand() restores the network's 16)."""
    n = N // 2
    rng = np.random.default_rng(seed)
    surr = B.Surrogate(n)
    xs, ys, states = [], [], []
    fa = torch.empty((n ** 3, 16), dtype=torch.float32, device=device)
    fb = torch.empty_like(fa)
    for r in range(n_rollouts):
        solid = leaf_mask(N, seed * 100003 + r, device)
        d = inlet_direction(rng)
        u_in = tuple(U_REF * d)
        surr.set_inlet(u_in if inlet_features else (0.0, 0.0, 0.0))
        lbm = B.LBM((N, N, N), tau, u_inlet=u_in, bc_x=1, max_tape=1)
        f = lbm.lattice(device)
        t = 0
        if rng.random() < turn_frac:
            t_turn = int(rng.integers(t_lo, t_hi)) // 2 * 2
            lbm.step(f, solid, t_turn)
            lbm.close()
            u_in = tuple(U_REF * turned(d, turn_deg, rng))
            surr.set_inlet(u_in if inlet_features else (0.0, 0.0, 0.0))
            lbm = B.LBM((N, N, N), tau, u_inlet=u_in, bc_x=1, max_tape=1)
            t = t_turn
            times = sorted(t_turn + int(x) // 2 * 2 for x in rng.integers(0, turn_window, per_rollout))
        else:
            times = sorted(int(x) // 2 * 2 for x in rng.integers(t_lo, t_hi, per_rollout))
        for t0 in times:
            if t0 < t:  # two draws closer than one block: skip the repeat
                continue
            lbm.step(f, solid, t0 - t)
            surr.features(f, solid, IN_SCALE, fa)
            if keep_states:
                states.append((f.clone(), solid, u_in))
            lbm.step(f, solid, block)
            t = t0 + block
            surr.features(f, solid, IN_SCALE, fb)
            xs.append(fa[:, :X_CH].clone())
            # du: channels 1-3 of the features (the reference velocity cancels)
            ys.append(((fb[:, 1:4] - fa[:, 1:4]) / IN_SCALE / OUT_SCALE).contiguous())
        lbm.close()
    surr.close()
    if keep_states:
        return xs, ys, states
    return xs, ys


def expand(a, width=16):
    """A compact [nv][k] pair array padded with zero channels to [nv][width]."""
    out = torch.zeros((a.shape[0], width), dtype=a.dtype, device=a.device)
    out[:, :a.shape[1]] = a
    return out


def init_params(nparams_slices, seed=0, device="cuda"):
    """He-style initial weights, zero biases, in the library's packing."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    total = nparams_slices[-1][1].stop
    p = torch.zeros(total, dtype=torch.float32)
    for ws, bs, cin, cout in nparams_slices:
        p[ws] = torch.randn(ws.stop - ws.start, generator=g) * math.sqrt(2.0 / (27 * cin))
    return p.to(device)


def layer_slices():
    ch = (16, 32, 32, 32, 16)
    out, o = [], 0
    for l in range(4):
        nw = 27 * ch[l] * ch[l + 1]
        out.append((slice(o, o + nw), slice(o + nw, o + nw + ch[l + 1]), ch[l], ch[l + 1]))
        o += nw + ch[l + 1]
    return out


def train(surr: B.Surrogate, xs, ys, steps, lr=1e-3, seed=0, log_every=0):
    """Adam over random training pairs; returns the loss of each step."""
    rng = np.random.default_rng(seed)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    for step in range(1, steps + 1):
        i = int(rng.integers(len(xs)))
        cur_lr = lr * 0.5 * (1.0 + math.cos(math.pi * step / steps))  # cosine decay
        loss.zero_()
        surr.set_features(expand(xs[i]) if xs[i].shape[1] < 16 else xs[i])
        surr.forward()
        surr.loss(expand(ys[i]) if ys[i].shape[1] < 16 else ys[i], loss)
        surr.backward()
        surr.adam(cur_lr, step)
        if log_every and step % log_every == 0:
            hist.append((step, loss.item()))
    return hist


def weights_path(N):
    return os.path.join(WEIGHTS_DIR, f"surrogate_lbm{N}.npy")


def load_weights(surr: B.Surrogate, N, device="cuda"):
    p = torch.from_numpy(np.load(weights_path(N)).astype(np.float32)).to(device)
    surr.set_params(p)


class SurrogateLBM:
    """Plain LBM plus the surrogate for blocks of BLOCK steps, with the check.

    Between surrogate calls the state is the fine (rho, u) field kept in the
    surrogate handle (chained mode); the lattice is re-initialised from it,
    f = f_eq(rho, u), only when the plain LBM takes over or at the end.

    inlet_features: give the network its features relative to the inlet
    velocity (surr_set_inlet); the shipped 128^3 weights were trained without
    (reference velocity zero). correct: add the last check's plain-minus-
    surrogate difference to every later block (surr_set_correction; measured
    to make the run worse, kept off by default). persistence: the scheme
    without the network, for comparison.

    use_graph replays each chained block from a CUDA graph; the default
    launches eagerly, which chains every kernel to the previous one by
    programmatic dependent launch, across blocks too."""

    def __init__(self, N, tau=0.55, u_inlet=(U_REF, 0.0, 0.0), check_every=3, tol=0.02,
                 params=None, device="cuda", use_graph=False, correct=False,
                 inlet_features=False, persistence=False):
        self.N = N
        self.lbm = B.LBM((N, N, N), tau, u_inlet=u_inlet, bc_x=1, max_tape=1)
        self.surr = B.Surrogate(N // 2)
        self.surr.set_inlet(u_inlet if inlet_features else (0.0, 0.0, 0.0))
        if params is None:
            load_weights(self.surr, N, device)
        else:
            self.surr.set_params(params)
        self.check_every, self.tol = check_every, tol
        self.calls = 0
        self.fallback = False
        self.errors = []
        self._sums = torch.zeros(2, dtype=torch.float64, device=device)
        self.use_graph = use_graph
        self.correct = correct
        # the same scheme without the network: every surrogate block keeps the
        # velocity unchanged (du = 0), for comparison
        self.persistence = persistence
        self._corr_on = False
        self._graphs = {}  # solid mask pointer -> CUDA graph of one chained block
        self._warm = set()

    # one block from a lattice (reads f, writes f)
    def surrogate_block(self, f, solid):
        """Advance f by BLOCK lattice steps with one network call (in place)."""
        self.surr.features(f, solid, IN_SCALE)
        self.surr.forward(keep_activations=False)
        self.surr.apply(solid, f, None, OUT_SCALE)
        return f

    # one block of the chained mode: the coarse features of the current fine
    # state are in the handle (from surr.features or the previous block);
    # the network runs and the fine state advances, leaving the features of
    # the new state for the next block
    def chained_block(self, solid):
        if self.persistence:
            return
        if not self.use_graph:
            self._chained_eager(solid)
            return
        key = solid.data_ptr() if solid is not None else 0
        g = self._graphs.get(key)
        if g is None:
            if key not in self._warm:
                # the first block runs eagerly, which also sets the kernels'
                # launch attributes outside any capture
                self._warm.add(key)
                self._chained_eager(solid)
                return
            # later blocks replay one captured block (capturing runs nothing)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self._chained_eager(solid)
            self._graphs[key] = g
        g.replay()

    def _chained_eager(self, solid):
        self.surr.forward(keep_activations=False)
        self.surr.advance_fine(OUT_SCALE, solid, IN_SCALE)

    def plain_block(self, f, solid):
        return self.lbm.step(f, solid, BLOCK)

    def velocity_error(self, f, g, solid):
        self._sums.zero_()
        B.lbm_velocity_error(f, g, solid, self._sums)
        e, r = self._sums.tolist()
        return math.sqrt(e / max(r, 1e-300))

    def fine_error(self, g, solid):
        self._sums.zero_()
        self.surr.fine_velocity_error(g, solid, self._sums)
        e, r = self._sums.tolist()
        return math.sqrt(e / max(r, 1e-300))

    def advance(self, f, solid, n_blocks):
        """n_blocks blocks of BLOCK steps on lattice f (in place); returns the
        number of blocks whose result came from the surrogate.

        Every check_every-th block is a check block: the fine state is taken
        from the lattice, the plain LBM advances the lattice, the surrogate
        advances the fine state, and the fluid velocities are compared; the
        run continues from the plain lattice. Other blocks chain the
        surrogate on the fine state; the lattice is rebuilt from it,
        f = f_eq(rho, u), only before a check block or at the end."""
        used = 0
        in_fine = False  # the current state is the handle's fine field, not f
        self.lbm.cache_mask(solid)  # the plain blocks share the mask's link words
        for _ in range(n_blocks):
            if self.fallback:
                self.plain_block(f, solid)
                continue
            if self.calls % self.check_every == 0:
                if in_fine:
                    self.surr.write_lattice(solid, f)
                    in_fine = False
                self.surr.features(f, solid, IN_SCALE)
                self.plain_block(f, solid)
                self.chained_block(solid)
                err = self.fine_error(f, solid)
                self.errors.append(err)
                if err > self.tol:
                    self.fallback = True
                elif self.correct:
                    # the plain block's difference from the surrogate's block is
                    # added to every later surrogate block (defect correction)
                    self.surr.set_correction(f, solid, 2 if self._corr_on else 1)
                    self._corr_on = True
            else:
                if not in_fine:
                    self.surr.features(f, solid, IN_SCALE)
                    in_fine = True
                self.chained_block(solid)
                used += 1
            self.calls += 1
        if in_fine:
            self.surr.write_lattice(solid, f)
        return used

    def reset(self):
        """Forget the check history and the correction (a new run)."""
        self.calls, self.errors, self.fallback = 0, [], False
        if self._corr_on:
            self.surr.set_correction(None, None, 0)
            self._corr_on = False

    def close(self):
        self.lbm.close()
        self.surr.close()
