"""Splitting one transform over several GPUs by Q (one process per GPU, torch.distributed).

Every (Q, segment) or (Q, face) pair is independent and each Q's sum is over all of the shape,
so the Q rows split into contiguous slabs, one per rank, with no exchange while the pairs are
summed.  The only collectives are the ones a caller asks for afterwards:

* the forward result: each rank holds its own slab; ``gather=True`` assembles all slabs on every
  rank (one all-gather of the per-rank results, padded to the longest slab);
* the vertex gradient: each rank's adjoint covers only its Q slab, and the gradient is their sum
  over ranks (one all-gather of the per-rank gradients, then a sum in rank order, so that every
  rank gets the same, reproducible result);
* the Q-gradient needs none: each rank owns the Q rows it differentiates.

Slabs start at multiples of ``align`` Q rows (the Q points one block of the main kernel holds:
4 per thread x 128 threads in 3D by default), so that each warp groups the same Q points as on one
GPU.  The per-rank work is a library call on the rank's own device; this module only partitions
and gathers, and its host logic is tested with CPU (gloo) ranks.
"""
from __future__ import annotations

DEFAULT_ALIGN = 512


def q_slab(n_q: int, rank: int, world: int, align: int = DEFAULT_ALIGN) -> tuple[int, int]:
    """[start, stop) of the Q rows owned by ``rank`` out of ``world``: contiguous, disjoint, covering
    0..n_q, each start a multiple of ``align`` (the last slab takes the remainder), slab sizes in
    units of ``align`` differing by at most one."""
    if world < 1 or not 0 <= rank < world or n_q < 0 or align < 1:
        raise ValueError("q_slab: need world >= 1, 0 <= rank < world, n_q >= 0, align >= 1")
    units = -(-n_q // align)
    base, extra = divmod(units, world)
    u0 = rank * base + min(rank, extra)
    u1 = u0 + base + (1 if rank < extra else 0)
    return min(n_q, u0 * align), min(n_q, u1 * align)


def _dist(group):
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def gather_slabs(local, n_q: int, align: int = DEFAULT_ALIGN, group=None):
    """All slabs of a per-Q result (rows = this rank's Q slab) in Q order, on every rank."""
    import torch
    import torch.distributed as dist
    rank, world = _dist(group)
    if world == 1:
        return local
    sizes = [q_slab(n_q, r, world, align) for r in range(world)]
    longest = max(b - a for a, b in sizes)
    pad = torch.zeros((longest,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[:local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:b - a] for p, (a, b) in zip(parts, sizes)], dim=0)


def sum_over_ranks(local, group=None):
    """Sum of a tensor over ranks, added in rank order on every rank (reproducible)."""
    import torch
    import torch.distributed as dist
    rank, world = _dist(group)
    if world == 1:
        return local
    parts = [torch.empty_like(local) for _ in range(world)]
    dist.all_gather(parts, local.contiguous(), group=group)
    total = parts[0].clone()
    for p in parts[1:]:
        total += p
    return total


def ft3d_q_sharded(verts, faces, q, *, options=None, gather=True, align=DEFAULT_ALIGN, group=None):
    """pft3d_mesh over this rank's Q slab (q holds all n_q rows on every rank); returns all rows
    (gather=True) or this rank's slab and its [start, stop)."""
    import paper_2104_08309_gb300 as pft
    rank, world = _dist(group)
    a, b = q_slab(q.shape[0], rank, world, align)
    local = pft.pft3d_mesh(verts, faces, q[a:b].contiguous(), options=options)
    return gather_slabs(local, q.shape[0], align, group) if gather else (local, (a, b))


def backward3d_q_sharded(verts, faces, q, grad_out, *, options=None, align=DEFAULT_ALIGN, group=None):
    """Vertex gradient sum_Q Re(conj(g) dF/dv) with the Q rows split over ranks: each rank runs the
    adjoint on its slab of q / grad_out (all n_q rows given on every rank), then the per-rank
    gradients are summed in rank order."""
    import torch
    import paper_2104_08309_gb300 as pft
    rank, world = _dist(group)
    a, b = q_slab(q.shape[0], rank, world, align)
    local = pft.pft3d_mesh_backward(verts, faces, q[a:b].contiguous(), grad_out[a:b].contiguous(), options=options)
    return sum_over_ranks(local.to(torch.float64), group).to(torch.float32)
