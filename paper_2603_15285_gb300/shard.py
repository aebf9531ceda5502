"""Data-parallel sharding of independent particles across ranks.

Particles are independent units (every step of the alignment is per particle),
so a run on N GPUs gives each rank its own contiguous range of particles and
needs no collective on the data path: only the timing barrier and the
max-over-ranks of the elapsed time, which these helpers provide.  A batch of
uneven particles is split by cost instead (longest processing time first);
the gradient of a template shared by all particles is the one real exchange,
a single sum over ranks.  The same helpers run on the ``nccl`` backend (CUDA
tensors) and on ``gloo`` (CPU).
"""


def dist_env():
    """(world_size, rank, local_rank) from the torchrun environment."""
    import os
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_start(rank: int, per_rank: int) -> int:
    """First particle index of `rank` when every rank aligns `per_rank` particles."""
    return rank * per_rank


def barrier(world_size: int):
    if world_size > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value: float, world_size: int, device="cpu") -> float:
    """The largest `value` over all ranks (the slowest rank's time)."""
    if world_size == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world_size: int, per_rank: int, seconds: float) -> float:
    """Whole-job throughput: all ranks' particles over the slowest rank's time."""
    return world_size * per_rank / seconds


def wigner_terms(L: int) -> int:
    """Wigner-D terms of one evaluation of C_L: sum_{l<=L} (2l+1)^2 (Appendix A.5)."""
    return (L + 1) * (2 * L + 1) * (2 * L + 3) // 3


def particle_cost(P: int, L_sched) -> int:
    """Refinement work of one particle: 3 P sum_j T(L_j) Wigner terms (about three
    evaluations per level and candidate); the dominant step of the path."""
    return 3 * int(P) * sum(wigner_terms(int(L)) for L in L_sched)


def lpt_shards(costs, world_size: int):
    """Longest processing time first: particles in decreasing cost (ties by
    index) each go to the rank with the smallest load so far (ties to the
    lower rank).  Returns one sorted index list per rank."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0] * world_size
    out = [[] for _ in range(world_size)]
    for i in order:
        r = min(range(world_size), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(s) for s in out]


def allreduce_sum(t, world_size: int):
    """Sum of a tensor over all ranks, in place (the template gradient of a
    template shared by every rank's particles)."""
    if world_size > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t
