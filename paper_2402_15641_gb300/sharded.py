"""The transform split by sensor column across ranks (one process per GPU).

Sec. 2: the second-plane matrix A^{3,4} (A2) is the same for every sensor
column, and the first-plane rows of column j involve column j alone.  So the
forward shards by column with no exchange: the rank holding columns
[j0, j1) builds a plan for that block (its A1 rows and the whole A2) and
computes p[:, j0:j1].  The adjoint A^T p is a sum over columns of each
column's share, so every rank applies its block's adjoint to p[:, j0:j1] and
one all-reduce (sum) of the volume gives A^T p on every rank.

A block plan computes its columns' angles exactly as the whole aperture's
plan does (srt_geometry.n_phi_total / phi_first), so a rank's forward is
bitwise the full forward's rows of its columns; the all-reduced adjoint sums
the same terms in another order (FP32 rounding apart).

The operator of a block is a factory argument: `Plan` by default (CUDA,
collectives over NCCL), or any object with forward(f) / adjoint(p) on torch
tensors, which is how the host logic is tested on CPU gloo ranks.
"""
from __future__ import annotations

from typing import Callable, Optional, Tuple

import torch


def column_range(n_phi: int, rank: int, world: int) -> Tuple[int, int]:
    """Columns [j0, j1) of `rank` when n_phi columns are split over `world`
    ranks as evenly as possible (the first n_phi % world ranks hold one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of {world}")
    if n_phi < world:
        raise ValueError(f"{n_phi} sensor columns cannot be split over {world} ranks")
    base, extra = divmod(n_phi, world)
    j0 = rank * base + min(rank, extra)
    return j0, j0 + base + (1 if rank < extra else 0)


class ColumnShard:
    """This rank's block of sensor columns and its operator.

    geom: the whole aperture's Geometry (srt.Geometry).
    make_op(geom, j0, j1): the block's operator; default: srt.Plan of
      geom.column_block(j0, j1) on the current CUDA device.
    group: torch.distributed process group (None: the default group; with
      no initialised group the shard is the whole aperture on one rank).
    """

    def __init__(self, geom, make_op: Optional[Callable] = None, group=None):
        import torch.distributed as dist
        self.geom = geom
        self.group = group
        dist_on = dist.is_available() and dist.is_initialized()
        self.world = dist.get_world_size(group) if dist_on else 1
        self.rank = dist.get_rank(group) if dist_on else 0
        self.j0, self.j1 = column_range(geom.n_phi, self.rank, self.world)
        if make_op is None:
            from .srt import Plan

            def make_op(g, j0, j1):
                return Plan(g.column_block(j0, j1) if (j0, j1) != (0, g.n_phi) else g)
        self.op = make_op(geom, self.j0, self.j1)

    @property
    def columns(self) -> int:
        return self.j1 - self.j0

    def forward(self, f: torch.Tensor) -> torch.Tensor:
        """p[..., j0:j1, :, :] of the whole forward, [B, j1 - j0, n_zs, n_ell]
        (or without B); no communication."""
        return self.op.forward(f)

    def gather(self, p_local: torch.Tensor) -> torch.Tensor:
        """The whole p on every rank from the ranks' blocks (all-gather)."""
        if self.world == 1:
            return p_local
        import torch.distributed as dist
        batched = p_local.dim() == 4
        pl = p_local if batched else p_local.unsqueeze(0)
        blocks = [column_range(self.geom.n_phi, r, self.world) for r in range(self.world)]
        cmax = max(j1 - j0 for j0, j1 in blocks)  # blocks padded to one size
        buf = torch.zeros((pl.shape[0], cmax, *pl.shape[2:]), dtype=pl.dtype, device=pl.device)
        buf[:, :self.columns] = pl
        parts = [torch.empty_like(buf) for _ in blocks]
        dist.all_gather(parts, buf, group=self.group)
        p = torch.cat([t[:, :j1 - j0] for t, (j0, j1) in zip(parts, blocks)], dim=1)
        return p if batched else p[0]

    def adjoint(self, p_local: torch.Tensor) -> torch.Tensor:
        """A^T p on every rank from this rank's columns p[..., j0:j1, :, :]:
        the block's adjoint, then one all-reduce (sum) of the volume."""
        f = self.op.adjoint(p_local)
        if self.world > 1:
            import torch.distributed as dist
            dist.all_reduce(f, op=dist.ReduceOp.SUM, group=self.group)
        return f

    def close(self):
        if hasattr(self.op, "close"):
            self.op.close()
