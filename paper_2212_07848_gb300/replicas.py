"""Host-side plumbing of replica parallelism (one process per GPU, independent
lattices, no data-path collective): the per-rank seed, the barrier around a
timed region and the whole-job rate from the slowest rank's time.  The only
collectives are these host-side reductions of timings; they run on whatever
process group the caller initialised (NCCL on GPUs, gloo in the CPU tests).
"""
import os


def rank_info(default_world=1):
    """(rank, world, local_rank) from the torchrun environment."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(default_world)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local_rank


def replica_seed(base_seed, rank):
    """Each rank runs its own replica: distinct Philox keys per rank."""
    return int(base_seed) + int(rank)


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest of one float per rank (the identity without a group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds_max):
    """Units processed by all ranks per second of the slowest rank."""
    if seconds_max <= 0:
        raise ValueError("timed region must be positive")
    return units_per_rank * world / seconds_max
