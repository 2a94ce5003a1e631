"""Index-range sharding over ranks: the paper's static division of the wanted
eigenpairs among processes (Sec. 3.1.2), one slice per GPU.

Each rank solves slice ``rank`` of ``world`` equal contiguous slices of
il..iu with ``api.eigh_tridiagonal_slice``: the root representation is
computed redundantly on every rank, a cluster that reaches across a slice
boundary is computed whole by both ranks that hold its members, and each
rank writes only its own columns of Z.  No data moves between ranks on the
solve path; the only collective is the optional gather of W (k doubles).

    res = shard.eigh_tridiagonal_sharded(d, e)          # inside torch.distributed
    res.W_local, res.Z_local, res.first, res.last, res.W   # W: all ranks' eigenvalues

The rank's slice and the gather are host logic on top of the C ABI; the
solve itself is the library's.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import api


@dataclass
class ShardResult:
    W_local: torch.Tensor        # eigenvalues first..last of this rank (ascending)
    Z_local: torch.Tensor | None  # their vectors, n x (last - first + 1)
    first: int                    # 1-based index range of this rank's slice
    last: int
    W: torch.Tensor | None        # every rank's eigenvalues in index order (gather_w), on this rank's device


def rank_and_world(group=None) -> tuple[int, int]:
    """(rank, world size) of torch.distributed's group, (0, 1) when it is not
    initialised."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


def gather_slices(W_local: torch.Tensor, world: int, group=None) -> torch.Tensor:
    """All ranks' W slices concatenated in rank order (slices differ in length
    by at most one: each is padded to the longest for all_gather)."""
    if world == 1:
        return W_local
    import torch.distributed as dist
    k = torch.tensor([W_local.numel()], dtype=torch.int64, device=W_local.device)
    ks = [torch.zeros_like(k) for _ in range(world)]
    dist.all_gather(ks, k, group=group)
    kmax = int(max(int(x) for x in ks))
    buf = torch.zeros(kmax, dtype=W_local.dtype, device=W_local.device)
    buf[:W_local.numel()] = W_local
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[:int(kk)] for p, kk in zip(parts, ks)])


def eigh_tridiagonal_sharded(d: torch.Tensor, e: torch.Tensor, il: int | None = None, iu: int | None = None, *,
                             group=None, margin: int = 32, vectors: bool = True, gather_w: bool = True,
                             plan: api.Plan | None = None) -> ShardResult:
    """This rank's slice of eigenpairs il..iu (default all) of the
    tridiagonal (d, e), which every rank holds whole; with ``gather_w`` the
    eigenvalues of all slices are gathered into W on every rank."""
    rank, world = rank_and_world(group)
    n = d.numel()
    il = 1 if il is None else int(il)
    iu = n if iu is None else int(iu)
    out = api.eigh_tridiagonal_slice(d, e, il, iu, world, rank, margin=margin, vectors=vectors, plan=plan)
    if vectors:
        W, Z, (a, b) = out
    else:
        (W, (a, b)), Z = out, None
    Wall = gather_slices(W, world, group) if gather_w else None
    return ShardResult(W_local=W, Z_local=Z, first=a, last=b, W=Wall)
