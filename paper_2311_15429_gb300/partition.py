"""Source partition across processes (one GPU each): who owns which domain,
and the one exchange of a step.

Sec. IV runs one process per domain: each computes its own domain's
contributions to the potentials of every domain, and each domain then
collects the contributions meant for it.  Here a rank owns a set of source
domains (``rp_own_sources``): its context keeps only their histories and its
``rp_evaluate`` writes, for every target domain, the sum over its owned
sources.  A target's total is then the sum of every rank's partial field for
it, delivered to the rank that owns the target by one reduce-scatter of
the packed partial fields: ``pack`` lays each rank's targets out in the
chunk of their owner, ``exchange`` sums the chunks across ranks and leaves
each rank its own, ``unpack`` splits it into its domains.  No arithmetic of
the method happens here: the sums are the exchange itself.
"""
from __future__ import annotations

from typing import Dict, List, Sequence


def owners(sizes: Sequence[int], world: int) -> List[int]:
    """Owner rank of each domain: the largest domains first, each to the rank
    with the fewest grid points so far (ties to the lower rank), so that the
    ranks' shares of the work and of the output are close."""
    load = [0] * world
    own = [0] * len(sizes)
    for d in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda k: (load[k], k))
        own[d] = r
        load[r] += sizes[d]
    return own


def owned_by(rank: int, own: Sequence[int]) -> List[int]:
    return [d for d, r in enumerate(own) if r == rank]


def chunk_floats(sizes: Sequence[int], own: Sequence[int], world: int) -> int:
    """Floats of one rank's chunk: the largest over ranks of 4 N summed over
    its domains (phi, Ax, Ay, Az per node)."""
    return max([sum(4 * sizes[d] for d, r in enumerate(own) if r == k) for k in range(world)] + [1])


def pack(fields, sizes: Sequence[int], own: Sequence[int], world: int):
    """fields[d]: the [4 N_d] partial field of domain d (a torch tensor, phi
    then A).  Returns the flat [world * chunk] buffer with domain d in its
    owner's chunk (domains of a chunk in id order, zero padding after)."""
    import torch
    C = chunk_floats(sizes, own, world)
    flat = torch.zeros(world * C, dtype=fields[0].dtype, device=fields[0].device)
    off = [k * C for k in range(world)]
    for d in range(len(sizes)):
        r = own[d]
        flat[off[r]:off[r] + 4 * sizes[d]] = fields[d].reshape(-1)
        off[r] += 4 * sizes[d]
    return flat


def exchange(flat, world: int, group=None):
    """Sum the packed buffers of every rank and keep this rank's chunk: a
    reduce-scatter (an all-reduce and the rank's slice where the backend has
    no reduce-scatter, e.g. gloo)."""
    import torch
    import torch.distributed as dist
    C = flat.numel() // world
    rank = dist.get_rank(group)
    if dist.get_backend(group) == "nccl":
        out = torch.empty(C, dtype=flat.dtype, device=flat.device)
        dist.reduce_scatter_tensor(out, flat, op=dist.ReduceOp.SUM, group=group)
        return out
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    return flat[rank * C:(rank + 1) * C].clone()


def unpack(chunk, rank: int, sizes: Sequence[int], own: Sequence[int]) -> Dict[int, object]:
    """The rank's chunk split into {domain: [4 N_d] total field}."""
    out, off = {}, 0
    for d in owned_by(rank, own):
        out[d] = chunk[off:off + 4 * sizes[d]]
        off += 4 * sizes[d]
    return out
