"""Column sharding over ranks.

The columns of one solve evolve independently (the Hamiltonian is shared and
read-only), so a solve splits into contiguous column blocks, one per rank.  The
only exchange is one sum over ranks of a few scalars after the forward pass
(the overlap terms that F and the co-state need) and one sum of the gradient
vectors at the end.  With one GPU per box, bench.py runs weak-scaled replicas;
these helpers carry the partition and the sums of the sharded form.
"""


def column_block(ncols, rank, world):
    """[start, stop) of rank's contiguous block of columns (sizes differ by <= 1)."""
    base, extra = divmod(ncols, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def allreduce_sum(tensor, group=None):
    """In-place sum over ranks of a float64 tensor (overlap terms or gradients)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(tensor, op=dist.ReduceOp.SUM, group=group)
    return tensor


def allreduce_max(value, device="cpu", group=None):
    """Max over ranks of a host float (the bench's timed-region duration)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
