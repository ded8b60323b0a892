"""Forward MPM rollouts through mpm_rollout, recorded once as a CUDA graph.

mpm_rollout runs all substeps of a rollout in one library call (re-sorting
the particles every `sort_every` substeps and fusing the G2P of each substep
with the P2G of the next); this class owns the state buffers, records that
call in a CUDA graph after a first eager run, and replays it.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import binding as B


class Rollout:
    def __init__(self, mpm: B.MPM, n: int, wind: B.WindField, n_substeps: int, *, t0: float = 0.0,
                 sort_every: int = 20, with_pins: bool = False, use_graph: bool = True,
                 device="cuda"):
        if n_substeps < 1 or sort_every < 0:
            raise ValueError("n_substeps must be >= 1 and sort_every >= 0")
        self.mpm, self.n, self.wind = mpm, n, wind
        self.n_substeps, self.t0, self.sort_every = n_substeps, t0, sort_every
        self.state = B.MpmState(*(torch.empty((r, n), dtype=torch.float32, device=device)
                                  for r in (3, 3, 9, 9)))
        self.pins = torch.zeros(n, dtype=torch.uint8, device=device) if with_pins else None
        self.ids = torch.empty(n, dtype=torch.int32, device=device)
        self.ids0 = torch.arange(n, dtype=torch.int32, device=device)
        self.use_graph = use_graph
        self.graph = None

    @property
    def kernel_launches(self):
        """Kernels of one run: one P2G, a grid update per substep, a fused
        G2P+P2G per substep but the last, one G2P, and per sort (at the start
        and every sort_every substeps) a scan of the 64 nb^3 cell counters
        (nb = ceil(n_grid / 4): two kernels for at most 1024 scan blocks of
        8192 counters, else three) and the scatter-move kernel, plus the key
        kernel for the first sort (and for every sort with the one-particle
        fused kernel; the paired one counts the keys itself)."""
        if self.n_substeps == 0:
            return 0
        sorts = -(-self.n_substeps // self.sort_every) if self.sort_every > 0 else 0
        nb = (self.mpm.n_grid + 3) // 4
        scan_blocks = -(-64 * nb ** 3 // 8192)
        per_sort = 1 + (2 if scan_blocks <= 1024 else 3)
        paired = getattr(self.mpm, "p2g_mode", B.P2G_AUTO) in (B.P2G_AUTO, B.P2G_PAIR)
        key_kernels = min(sorts, 1) if paired else sorts
        return 1 + 2 * self.n_substeps + per_sort * sorts + key_kernels

    def _issue(self):
        self.mpm.rollout(self.state, self.pins, self.ids, self.wind, self.t0, self.n_substeps,
                         self.sort_every)

    def _capture(self):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=s):
            self._issue()
        torch.cuda.current_stream().wait_stream(s)

    def load(self, state: B.MpmState, pinned: Optional[torch.Tensor] = None):
        """Copy an initial state (and pin flags) into the rollout's buffers."""
        for dst, src in zip(self.state, state):
            dst.copy_(src, non_blocking=True)
        self.ids.copy_(self.ids0, non_blocking=True)
        if self.pins is not None:
            if pinned is None:
                self.pins.zero_()
            else:
                self.pins.copy_(pinned, non_blocking=True)

    def run(self):
        """Advance the loaded state. The first call runs eagerly (which also
        loads every kernel) and then records the graph that later calls replay."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self._issue()
            if self.use_graph:
                self._capture()
        return self.result()

    def result(self):
        """(final state in sorted order, ids: original index of each particle)."""
        return self.state, self.ids
