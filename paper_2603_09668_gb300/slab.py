"""Host logic of one MLS-MPM scene split over ranks in slabs of grid layers.

A scene whose grid or particle set outgrows one GPU is cut along z, the
slowest axis of the node index (k N + j) N + i, so that every slab, and every
halo, is one contiguous range of grid memory. Rank r owns the node layers
k0 <= k < k1 and the particles whose stencil base layer
floor(z / dx - 1/2) (the first of the 3 layers the quadratic B-spline weights
of Eq. 4 reach) lies in that range when the particles are last assigned.

Per substep (Eq. 5 - Eq. 8):

1. P2G on the rank's own particles writes mass and momentum into layers
   [k0 - margin, k1 + 2 + margin): its own slab, 2 layers above it that the
   stencil reaches from base k1 - 1, and `margin` layers on each side for
   particles that drifted across the slab face since they were last assigned.
2. ``halo_sum``: each rank sends the partial sums in its ghost layers to the
   neighbour that owns them and adds what it receives into its own layers.
   After this every owned node holds the same mass and momentum as on one
   rank (up to the order of the floating-point additions).
3. The grid update (Eq. 6 - 7) runs on owned nodes only: it is local per node.
4. ``halo_fill``: each rank copies the updated velocities of its boundary
   layers into the neighbours' ghost layers, so that G2P of its own particles
   reads the full 3^3 stencil.
5. G2P and the deformation update (Eq. 8) of the rank's own particles.

Particles are re-assigned only where the sorted path re-sorts them (every
``sort_every`` substeps): ``migrate`` sends each particle whose base layer left
the rank's slab to the owner of that layer. Between re-sorts a particle may
drift at most `margin` cells in z (one cell per substep is the CFL bound of the
explicit update); ``check_drift`` verifies it before the next P2G.

Exchanges are plain point-to-point sends and receives between neighbouring
ranks (``torch.distributed`` isend / irecv: NCCL on GPU tensors, gloo on CPU
tensors), with no collective over all ranks and no multicast. Grid tensors are
[C][N][N][N] with the layer index k first after the channel, the layout of the
node index above.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Sequence

import numpy as np
import torch
import torch.distributed as dist

STENCIL_REACH = 2  # layers above the base layer that the quadratic weights touch


def layer_bounds(n_grid: int, world: int) -> list:
    """Even split of the n_grid node layers over `world` ranks: rank r owns
    [bounds[r], bounds[r + 1])."""
    if world < 1 or n_grid < world:
        raise ValueError(f"cannot split {n_grid} layers over {world} ranks")
    return [r * n_grid // world for r in range(world + 1)]


def base_layer(z: np.ndarray, n_grid: int) -> np.ndarray:
    """Stencil base layer floor(z n_grid - 1/2) of particles at height z."""
    return np.floor(np.asarray(z, np.float64) * n_grid - 0.5).astype(np.int64)


@dataclass(frozen=True)
class Slab:
    n_grid: int
    world: int
    rank: int
    margin: int = 1

    @property
    def bounds(self):
        return layer_bounds(self.n_grid, self.world)

    @property
    def k0(self):
        return self.bounds[self.rank]

    @property
    def k1(self):
        return self.bounds[self.rank + 1]

    @property
    def lo(self):
        """First layer this rank's P2G and G2P touch."""
        return max(self.k0 - self.margin, 0)

    @property
    def hi(self):
        """One past the last layer this rank's P2G and G2P touch."""
        return min(self.k1 + STENCIL_REACH + self.margin, self.n_grid)

    def validate(self):
        widths = np.diff(self.bounds)
        if widths.min() < STENCIL_REACH + self.margin:
            raise ValueError("a slab is thinner than the halo it has to serve")
        if self.margin < 0:
            raise ValueError("negative drift margin")

    def owner(self, z: np.ndarray) -> np.ndarray:
        """Rank that owns each particle's base layer (layers below 0 or above
        n_grid - 1 go to the first or last rank)."""
        b = np.clip(base_layer(z, self.n_grid), 0, self.n_grid - 1)
        return np.searchsorted(np.asarray(self.bounds[1:]), b, side="right")

    def check_drift(self, z: np.ndarray):
        """Raise if a particle's base layer left [k0 - margin, k1 + margin):
        its stencil would reach past the halo the exchanges keep."""
        b = base_layer(z, self.n_grid)
        lo = self.k0 - self.margin if self.rank > 0 else -(1 << 40)
        hi = self.k1 + self.margin if self.rank < self.world - 1 else (1 << 40)
        bad = np.flatnonzero((b < lo) | (b >= hi))
        if bad.size:
            raise RuntimeError(f"rank {self.rank}: {bad.size} particles drifted past the "
                               f"{self.margin}-layer margin; re-sort more often")


def _exchange(sends: Sequence, recvs: Sequence, group=None):
    """Post every send and receive ((peer, tensor) pairs) and wait for all."""
    reqs = [dist.irecv(t, src=p, group=group) for p, t in recvs]
    reqs += [dist.isend(t, dst=p, group=group) for p, t in sends]
    for r in reqs:
        r.wait()


def halo_sum(grid: torch.Tensor, slab: Slab, group=None):
    """Add the neighbours' partial P2G sums for this rank's layers into `grid`
    ([C][N][N][N], in place) and clear this rank's ghost layers. The upper
    ghost [k1, hi) goes to rank + 1, the lower ghost [lo, k0) to rank - 1."""
    r, W = slab.rank, slab.world
    sends, recvs, adds = [], [], []
    if r + 1 < W:
        up = Slab(slab.n_grid, W, r + 1, slab.margin)
        sends.append((r + 1, grid[:, slab.k1:slab.hi].contiguous()))
        buf = torch.empty_like(grid[:, up.lo:slab.k1])
        recvs.append((r + 1, buf))
        adds.append((up.lo, slab.k1, buf))
    if r > 0:
        dn = Slab(slab.n_grid, W, r - 1, slab.margin)
        sends.append((r - 1, grid[:, slab.lo:slab.k0].contiguous()))
        buf = torch.empty_like(grid[:, slab.k0:dn.hi])
        recvs.append((r - 1, buf))
        adds.append((slab.k0, dn.hi, buf))
    _exchange(sends, recvs, group)
    for a, b, buf in adds:
        grid[:, a:b] += buf
    grid[:, slab.lo:slab.k0] = 0
    grid[:, slab.k1:slab.hi] = 0


def halo_fill(grid: torch.Tensor, slab: Slab, group=None):
    """Copy the neighbours' owned values into this rank's ghost layers of
    `grid` (in place): [k1, hi) from rank + 1 and [lo, k0) from rank - 1."""
    r, W = slab.rank, slab.world
    sends, recvs = [], []
    if r + 1 < W:
        up = Slab(slab.n_grid, W, r + 1, slab.margin)
        sends.append((r + 1, grid[:, up.lo:slab.k1].contiguous()))
        recvs.append((r + 1, grid[:, slab.k1:slab.hi]))
    if r > 0:
        dn = Slab(slab.n_grid, W, r - 1, slab.margin)
        sends.append((r - 1, grid[:, slab.k0:dn.hi].contiguous()))
        recvs.append((r - 1, grid[:, slab.lo:slab.k0]))
    bufs = [(t, torch.empty_like(t)) for _, t in recvs]
    _exchange(sends, [(p, b) for (p, _), (_, b) in zip(recvs, bufs)], group)
    for dst, b in bufs:
        dst.copy_(b)


def migrate(particles: torch.Tensor, z_row: int, slab: Slab, group=None) -> torch.Tensor:
    """Re-assign particles to the owners of their base layers. `particles` is
    [R][n] (all per-particle rows stacked: x, v, C, F, pinned, ids ..., one
    dtype); row `z_row` holds z. Particles leaving go to rank - 1 or rank + 1
    (at most one slab per re-sort: the drift margin is thinner than a slab);
    arrivals are appended after the particles that stay. Returns the new
    [R][n'] tensor."""
    r, W = slab.rank, slab.world
    own = slab.owner(particles[z_row].cpu().numpy())
    if np.any(np.abs(own - r) > 1):
        raise RuntimeError(f"rank {r}: a particle skipped a whole slab")
    stay = torch.from_numpy(own == r).to(particles.device)
    peers = [p for p in (r - 1, r + 1) if 0 <= p < W]
    out = {p: particles[:, torch.from_numpy(own == p).to(particles.device)].contiguous()
           for p in peers}
    # counts first, then the particle rows
    cnt_in = {p: torch.zeros(1, dtype=torch.int64, device=particles.device) for p in peers}
    _exchange([(p, torch.tensor([out[p].shape[1]], dtype=torch.int64, device=particles.device))
               for p in peers], [(p, cnt_in[p]) for p in peers], group)
    R = particles.shape[0]
    bufs = {p: torch.empty((R, int(cnt_in[p])), dtype=particles.dtype, device=particles.device)
            for p in peers}
    _exchange([(p, out[p]) for p in peers if out[p].shape[1]],
              [(p, bufs[p]) for p in peers if bufs[p].shape[1]], group)
    return torch.cat([particles[:, stay]] + [bufs[p] for p in peers], dim=1)
