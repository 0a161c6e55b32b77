"""Row-strip domain decomposition of one large image over ranks: one halo exchange per iteration.

One iPiano step (Eq. iPianoupdate) at a pixel reads the iterate within 6 pixels of it: the gradient of the prior
(Eq. FoEF) there sums K_i^T psi_i over the responses within 3 pixels, and each response reads u within 3 more;
the inertial term and the prox are pointwise.  So a rank that owns the rows [r0, r1) of the image can compute
the next iterate of those rows from its rows plus HALO = 6 rows above and below, which its neighbours own.  It
holds an extended strip (its rows and the halo rows that exist); before every step it receives the halo rows of
the current iterate from its neighbours and sends them its own boundary rows (point-to-point, one message per
neighbour and direction); then it runs the ordinary single-image step on the extended strip and keeps its own
rows.  The extended strip's cut edges are treated by the step as image borders, which corrupts only rows within
6 of them: halo rows, which are discarded.  At the image's own top and bottom the strip edge is the image
border, where the padding P applies as in the single-image solve.  Every owned pixel therefore sees exactly the
arithmetic of the single-domain solve.

The data term, the initial iterate and the previous iterate are only read at owned pixels and need no
exchange.  Strips are balanced to within one row and must hold at least HALO rows, so that every halo row
comes from an adjacent rank.  The exchange uses torch.distributed point-to-point calls on torch tensors, so the
same code moves CPU tensors over gloo or device tensors over NCCL; the step is a callable on the extended strip.
"""
from __future__ import annotations

from typing import Callable

import torch

HALO = 6  # rows of the iterate that one step at a pixel reads on either side (3 for K_i, 3 for K_i^T)


def strip_rows(H: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [r0, r1) that `rank` owns: H split into `world` strips whose sizes differ by at most one."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    base, extra = divmod(H, world)
    if base < HALO:
        raise ValueError(f"{H} rows over {world} ranks leave strips below the halo of {HALO} rows")
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def extended_rows(H: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [e0, e1) of the extended strip: the owned rows and the halo rows that lie in the image."""
    r0, r1 = strip_rows(H, world, rank)
    return max(0, r0 - HALO), min(H, r1 + HALO)


def exchange_halo(u_ext: torch.Tensor, H: int, world: int, rank: int, dist) -> None:
    """Fills the halo rows of u_ext (rows [e0, e1) of the image) from the neighbouring ranks and sends them this
    rank's boundary rows.  Messages going up carry tag 0, messages going down tag 1."""
    r0, r1 = strip_rows(H, world, rank)
    e0, _ = extended_rows(H, world, rank)
    reqs, recvs = [], []
    if rank > 0:
        reqs.append(dist.isend(u_ext[r0 - e0:r0 - e0 + HALO].contiguous(), rank - 1, tag=0))
        top = torch.empty_like(u_ext[:HALO])
        reqs.append(dist.irecv(top, rank - 1, tag=1))
        recvs.append((slice(0, HALO), top))
    if rank < world - 1:
        reqs.append(dist.isend(u_ext[r1 - e0 - HALO:r1 - e0].contiguous(), rank + 1, tag=1))
        bottom = torch.empty_like(u_ext[:HALO])
        reqs.append(dist.irecv(bottom, rank + 1, tag=0))
        recvs.append((slice(r1 - e0, r1 - e0 + HALO), bottom))
    for r in reqs:
        r.wait()
    for rows, buf in recvs:
        u_ext[rows] = buf


StepFn = Callable[[torch.Tensor, torch.Tensor, torch.Tensor], torch.Tensor]


def solve_strip(step: StepFn, d_ext: torch.Tensor, u0_ext: torch.Tensor, iters: int, H: int, world: int,
                rank: int, dist) -> torch.Tensor:
    """Runs `iters` iPiano steps of the whole image, this rank computing its strip.

    step(d, u, u_prev) returns the next iterate of an image (here the extended strip) from the data term d, the
    iterate u and the previous iterate u_prev (Eq. iPianoupdate with u^{-1} = u^0 at the start).  d_ext and
    u0_ext are the extended strip's rows of the data term and of the initial iterate; only their owned rows are
    read.  Returns the owned rows of u^iters."""
    r0, r1 = strip_rows(H, world, rank)
    e0, e1 = extended_rows(H, world, rank)
    if d_ext.shape[0] != e1 - e0 or u0_ext.shape[0] != e1 - e0:
        raise ValueError(f"rank {rank}: extended strip has {e1 - e0} rows")
    own = slice(r0 - e0, r1 - e0)
    u = u0_ext.clone()
    u_prev = u.clone()
    for _ in range(iters):
        exchange_halo(u, H, world, rank, dist)
        u_next = step(d_ext, u, u_prev)
        u_prev[own] = u[own]
        u[own] = u_next[own]
    return u[own].clone()
