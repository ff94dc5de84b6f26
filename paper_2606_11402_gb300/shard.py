"""Sharding the factor, the NLL and its gradient over processes (one per GPU)
by contiguous ranges of graph positions.

Once the graph is built, the conditional of every point (Sec. 2.1 Eq. 2)
depends only on its own and its neighbours' coordinates, and whitening needs
only the field values of those neighbours; so the factor, xi = L^-1 v, the
log-determinant, the NLL and the NLL gradient split by position without any
exchange inside the computation.  Each process holds the whole graph (built
from the same points), factors its own range of positions
(graphgp_factor_rows), and per NLL evaluation:

1. all-gathers the field v (every rank contributes its own slice; the other
   slices are the halo its rows read -- with position ranges cut across the
   depth levels the halo of a range is most of the earlier ranges, so a full
   all-gather is the exchange),
2. evaluates its part of the NLL and of the gradient (graphgp_nll_rows,
   graphgp_nll_backward_rows),
3. sums the NLL parts and the theta_bar parts (all-reduce) and the vbar
   contributions, which land on its own positions and on its rows'
   neighbours (all-reduce), keeping its own slice.

Generation (v = L xi) is not split: every depth level would need an exchange.
Collectives go through torch.distributed (NCCL on GPUs, gloo on CPU); no
library kernel reads another GPU's memory.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist


def position_ranges(N: int, n0: int, world: int) -> list[tuple[int, int]]:
    """Contiguous [begin, end) ranges covering 0..N with about N / world
    positions each.  Range 0 starts at 0 and holds the dense block (it ends at
    or after n0); every other range starts at or after n0."""
    if world < 1:
        raise ValueError("world must be >= 1")
    cuts = [0]
    for r in range(1, world):
        c = int(round(r * N / world))
        cuts.append(min(N, max(c, n0, cuts[-1])))
    cuts.append(N)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


class GpuRowOps:
    """The compute of one range on this process's GPU through the C ABI."""

    def __init__(self, graph, kernel, p0: int, p1: int):
        from . import factor_rows
        self.graph = graph
        self.fac = factor_rows(graph, kernel, p0, p1)
        self.N = graph.N

    def nll(self, v_full: torch.Tensor) -> torch.Tensor:
        from . import nll_rows
        return nll_rows(self.graph, self.fac, v_full)

    def nll_backward(self, v_full: torch.Tensor):
        from . import nll_backward_rows
        vbar = torch.zeros_like(v_full)
        tb = torch.zeros(3, dtype=torch.float64, device=v_full.device)
        nll_backward_rows(self.graph, self.fac, v_full, vbar, tb)
        return vbar, tb


class ShardedNLL:
    """NLL(v; theta) and its gradient with the positions split over the
    processes of `group`.  `ops` computes one range (default: GpuRowOps on
    this process's GPU); tests pass a CPU stand-in."""

    def __init__(self, N: int, n0: int, ops_factory, group=None):
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.ranges = position_ranges(N, n0, self.world)
        self.p0, self.p1 = self.ranges[self.rank]
        self.N = N
        self.width = max(e - b for b, e in self.ranges)
        self.ops = ops_factory(self.p0, self.p1)

    def gather_field(self, v_own: torch.Tensor) -> torch.Tensor:
        """All ranks' slices of v into one full-length vector (slices padded
        to the widest range for the collective)."""
        if v_own.numel() != self.p1 - self.p0:
            raise ValueError("v_own must hold this rank's positions")
        pad = torch.zeros(self.width, dtype=v_own.dtype, device=v_own.device)
        pad[:v_own.numel()] = v_own
        parts = [torch.empty_like(pad) for _ in range(self.world)]
        dist.all_gather(parts, pad, group=self.group)
        return torch.cat([parts[r][:e - b] for r, (b, e) in enumerate(self.ranges)])

    def value_and_grad(self, v_own: torch.Tensor):
        """(NLL, dNLL/dv on this rank's positions, dNLL/d(l, s2, nugget))."""
        v_full = self.gather_field(v_own)
        part = self.ops.nll(v_full).to(torch.float64).reshape(1).clone()
        vbar, tb = self.ops.nll_backward(v_full)
        vbar = vbar.clone()
        tb = tb.to(torch.float64).reshape(3).clone()
        dist.all_reduce(part, group=self.group)
        dist.all_reduce(vbar, group=self.group)
        dist.all_reduce(tb, group=self.group)
        return part, vbar[self.p0:self.p1], tb


def halo_positions(nbr_pos: np.ndarray, n0: int, p0: int, p1: int) -> np.ndarray:
    """Positions outside [p0, p1) that the rows of [p0, p1) read (their
    neighbours), sorted: the halo of the range."""
    lo = max(p0, n0) - n0
    hi = max(p1 - n0, 0)
    if hi <= lo:
        return np.zeros(0, np.int64)
    c = np.unique(np.asarray(nbr_pos[lo:hi]).reshape(-1).astype(np.int64))
    return c[(c < p0) | (c >= p1)]
