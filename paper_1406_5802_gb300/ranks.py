"""Host-side bookkeeping for runs with one process per GPU (torchrun ranks).

The method's solves are independent problems, so N ranks run N replicas, each on its own system, and
no collective touches the data path.  The one exchange is the timing: the whole job lasts as long as
its slowest rank, so its rate is the units of all ranks over the maximum of the ranks' times.  Nothing
here runs on a GPU: the maximum goes through whatever backend the process group was created with
(NCCL for the benchmark, gloo in the CPU tests).
"""

SEED_STRIDE = 7919  # a prime: rank r draws its system from seed base + r * SEED_STRIDE


def system_seed(base: int, rank: int) -> int:
    """Seed of the system that `rank` solves: distinct for every rank, rank 0 keeps `base`."""
    if rank < 0:
        raise ValueError(f"rank must be >= 0, got {rank}")
    return base + SEED_STRIDE * rank


def max_over_ranks(value: float, world: int, device: str = "cpu") -> float:
    """The maximum of `value` over all ranks (`value` itself when world == 1, with no process group)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units per second of the whole job: every rank's units over the slowest rank's time."""
    if not seconds > 0.0:
        raise ValueError(f"the timed region must be positive, got {seconds}")
    return units_per_rank * world / seconds
