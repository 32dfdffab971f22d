"""Exchange step of a decomposition of one PSFD operator over several ranks (one GPU per rank).

The operator of Sec. 2.2 has two stages with different locality in the HYBRID (kx, ky, z)
domain: the axial stage (curl-curl with the stretched derivative, the PML, the multilayer
reflection R) needs whole z columns of every lateral mode, and the lateral contrast stage
(IFFT2, x deps, FFT2) needs whole z planes.  With the Krylov vectors distributed by lateral
columns (rank r owns the columns [c0_r, c1_r) of every plane), the axial stage is local and only
the absorber planes move: per apply, the axial stage's G = E + R E on the absorber planes goes
to a plane distribution (rank r owns planes [z0_r, z1_r) of the absorber range, every column),
the contrast stage runs plane by plane, and its result comes back to the column distribution
to be subtracted.  Dot products are local sums followed by one FP64 all-reduce.

`ColumnPlaneExchange` is that exchange for arrays of shape [lead][planes][columns] (lead = rhs x
components): `to_planes` sends every rank the planes it owns, restricted to each sender's
columns, and `to_columns` is the inverse.  It is a pure data movement over
torch.distributed.all_to_all_single and holds no arithmetic of the method.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import torch
import torch.distributed as dist


def even_split(n: int, parts: int) -> List[Tuple[int, int]]:
    """[start, stop) of `parts` nearly equal ranges covering 0 .. n - 1 (the first ones one longer)."""
    base, extra = divmod(n, parts)
    out, s = [], 0
    for p in range(parts):
        e = s + base + (1 if p < extra else 0)
        out.append((s, e))
        s = e
    return out


class ColumnPlaneExchange:
    """Column distribution <-> plane distribution of arrays [lead][planes][columns]."""

    def __init__(self, planes: int, columns: int, world: int, rank: int, group=None):
        self.planes, self.columns, self.world, self.rank, self.group = planes, columns, world, rank, group
        self.col = even_split(columns, world)
        self.pln = even_split(planes, world)

    def my_columns(self) -> Tuple[int, int]:
        return self.col[self.rank]

    def my_planes(self) -> Tuple[int, int]:
        return self.pln[self.rank]

    def to_planes(self, x_cols: torch.Tensor) -> torch.Tensor:
        """x_cols [lead][planes][my columns] -> [lead][my planes][columns]."""
        lead = x_cols.shape[0]
        c0, c1 = self.my_columns()
        assert x_cols.shape == (lead, self.planes, c1 - c0)
        # send block for rank s: my columns of rank s's planes, packed [s][lead][planes_s][my columns]
        send = torch.cat([x_cols[:, p0:p1, :].reshape(-1) for p0, p1 in self.pln])
        in_sizes = [lead * (p1 - p0) * (c1 - c0) for p0, p1 in self.pln]
        z0, z1 = self.my_planes()
        out_sizes = [lead * (z1 - z0) * (b1 - b0) for b0, b1 in self.col]
        recv = torch.empty(sum(out_sizes), dtype=x_cols.dtype, device=x_cols.device)
        dist.all_to_all_single(recv, send.contiguous(), out_sizes, in_sizes, group=self.group)
        parts = torch.split(recv, out_sizes)
        blocks = [parts[s].reshape(lead, z1 - z0, b1 - b0) for s, (b0, b1) in enumerate(self.col)]
        return torch.cat(blocks, dim=2)

    def to_columns(self, y_planes: torch.Tensor) -> torch.Tensor:
        """y_planes [lead][my planes][columns] -> [lead][planes][my columns] (inverse of to_planes)."""
        lead = y_planes.shape[0]
        z0, z1 = self.my_planes()
        assert y_planes.shape == (lead, z1 - z0, self.columns)
        send = torch.cat([y_planes[:, :, b0:b1].reshape(-1) for b0, b1 in self.col])
        in_sizes = [lead * (z1 - z0) * (b1 - b0) for b0, b1 in self.col]
        c0, c1 = self.my_columns()
        out_sizes = [lead * (p1 - p0) * (c1 - c0) for p0, p1 in self.pln]
        recv = torch.empty(sum(out_sizes), dtype=y_planes.dtype, device=y_planes.device)
        dist.all_to_all_single(recv, send.contiguous(), out_sizes, in_sizes, group=self.group)
        parts = torch.split(recv, out_sizes)
        blocks = [parts[s].reshape(lead, p1 - p0, c1 - c0) for s, (p0, p1) in enumerate(self.pln)]
        return torch.cat(blocks, dim=1)


def distributed_dot(local_sums: Sequence[float], group=None) -> torch.Tensor:
    """The FP64 all-reduce of the ranks' local dot-product sums (one per right-hand side)."""
    t = torch.tensor(list(local_sums), dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t
