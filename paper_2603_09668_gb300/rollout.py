"""Forward MPM rollouts: many substeps of one scene with periodic re-sorting of
the particles by grid cell, recorded once as a CUDA graph and replayed.

The graph holds, per segment of `sort_every` substeps, one mpm_sort (state
ping-pong, particle ids carried along) followed by in-place mpm_substep calls
at times t0 + k dt. Replaying it issues every kernel of the rollout with one
launch from the host.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import binding as B


class Rollout:
    def __init__(self, mpm: B.MPM, n: int, wind: B.WindField, n_substeps: int, *, t0: float = 0.0,
                 sort_every: int = 20, with_pins: bool = False, use_graph: bool = True,
                 device="cuda"):
        if n_substeps < 1 or sort_every < 1:
            raise ValueError("n_substeps and sort_every must be >= 1")
        self.mpm, self.n, self.wind = mpm, n, wind
        self.n_substeps, self.t0, self.sort_every = n_substeps, t0, sort_every
        self.dt = mpm.dt
        shapes = (3, 3, 9, 9)
        self.bufs = [B.MpmState(*(torch.empty((r, n), dtype=torch.float32, device=device)
                                  for r in shapes)) for _ in range(2)]
        self.pins = [torch.zeros(n, dtype=torch.uint8, device=device) for _ in range(2)] \
            if with_pins else [None, None]
        self.ids = [torch.empty(n, dtype=torch.int32, device=device) for _ in range(2)]
        self.n_sorts = (n_substeps + sort_every - 1) // sort_every
        self.final = self.n_sorts % 2  # buffer holding the result
        self.use_graph = use_graph
        self.graph = None

    # kernels per replay: the substeps (P2G, grid, G2P) and the sorts
    # (keys, 3 scan kernels, scatter, permute)
    @property
    def kernel_launches(self):
        return 3 * self.n_substeps + 6 * self.n_sorts

    def _issue(self):
        cur = 0
        for k in range(self.n_substeps):
            if k % self.sort_every == 0:
                nxt = 1 - cur
                ids_in = None if k == 0 else self.ids[cur]
                self.mpm.sort(self.bufs[cur], self.bufs[nxt], self.pins[cur], self.pins[nxt],
                              ids_in, self.ids[nxt])
                cur = nxt
            self.mpm.substep(self.bufs[cur], self.bufs[cur], self.pins[cur], self.wind,
                             self.t0 + k * self.dt)
        assert cur == self.final

    def _capture(self):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=s):
            self._issue()
        torch.cuda.current_stream().wait_stream(s)

    def load(self, state: B.MpmState, pinned: Optional[torch.Tensor] = None):
        """Copy an initial state (and pin flags) into the rollout's input buffer."""
        for dst, src in zip(self.bufs[0], state):
            dst.copy_(src, non_blocking=True)
        if self.pins[0] is not None:
            if pinned is None:
                self.pins[0].zero_()
            else:
                self.pins[0].copy_(pinned, non_blocking=True)

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
        return self.bufs[self.final], self.ids[self.final]
