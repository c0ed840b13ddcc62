"""Host side of running on several GPUs: one process per GPU, no data-path collective.

The method's problems are independent (one mesh, or a batch of meshes, per GPU), so a multi-GPU
run is a set of replicas (weak scaling) or a partition of a batch's meshes over the ranks.  The
only communication is host-side bookkeeping: a barrier around the timed region and the
reduction of the per-rank timings into one whole-job rate.  Nothing here touches the kernels.
"""


def shard(n, rank, world):
    """Contiguous, balanced share of n independent units (meshes of a batch) for `rank` out of
    `world`: the first n % world ranks take one unit more.  Returns a range."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"bad shard request: n={n}, rank={rank}, world={world}")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def whole_job_rate(units, ms, dist=None, device="cpu"):
    """Whole-job throughput of a timed region: the units all ranks processed divided by the
    slowest rank's time.  `units` and `ms` are this rank's; with `dist` (an initialised
    torch.distributed) they are summed / maxed over the ranks.  Returns (units per second,
    total units, max ms)."""
    if dist is None:
        total, slowest = float(units), float(ms)
    else:
        import torch
        t = torch.tensor([float(units)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        m = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        dist.all_reduce(m, op=dist.ReduceOp.MAX)
        total, slowest = float(t.item()), float(m.item())
    if not slowest > 0.0:
        raise ValueError(f"timed region of {slowest} ms")
    return total / (slowest / 1000.0), total, slowest
