"""Shot-parallel helpers for several processes (one GPU each).

The solves of different shots are independent (no exchange during time
stepping), so work is split by shots and only the results meet: gathers stay
with the rank that computed them, misfits and velocity gradients are summed
across ranks in FP64."""


def shard_shots(nshots, rank, world):
    """Contiguous shot range [lo, hi) of `rank` out of `world` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    base, extra = divmod(nshots, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def allreduce_fp64(tensor, group=None):
    """Sum a gradient or misfit over all ranks in FP64; returns the FP64 sum."""
    import torch
    import torch.distributed as dist
    t = tensor.detach().to(torch.float64).clone()
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        if dist.get_backend(group) == "nccl" and not t.is_cuda:
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t
