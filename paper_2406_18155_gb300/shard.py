"""Column sharding over ranks (the paper's distribution of the unitary's columns
across devices, Sec. 4.2).

The columns of one solve evolve independently (the Hamiltonian is shared and
read-only), so a solve splits into contiguous column blocks, one per rank.  The
fidelity couples them only through sums over columns: after the forward pass the
shards sum {Re z, Im z, q, S_c} (z = tr M, q = tr M M^dag, S_c the computational
columns), build their co-states from the totals, and at the end sum their
gradients.  `sg_fidelity_grad_sharded` performs both sums through a callback;
`torch_allreduce` builds that callback from a torch.distributed process group.
"""
import numpy as np


def column_block(ncols, rank, world):
    """[start, stop) of rank's contiguous block of columns (sizes differ by <= 1)."""
    base, extra = divmod(ncols, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def torch_allreduce(group=None, device="cpu"):
    """A sum over the ranks of `group` for the library's sharded solve: maps a float64
    numpy vector to its element-wise sum over ranks.  device "cpu" for gloo, a CUDA
    device for nccl (the vector is copied there and back)."""
    import torch
    import torch.distributed as dist

    def reduce(v):
        t = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).to(device)
        if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return t.cpu().numpy()
    return reduce


def allreduce_max(value, device="cpu", group=None):
    """Max over ranks of a host float (the bench's timed-region duration)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
