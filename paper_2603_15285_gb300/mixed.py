"""Batches that mix box sizes and bandwidths.

A plan is built for one (box, shells, schedule, P_max); a mixed batch is a
list of groups, each aligned with its own plan.  The groups are independent, so
each runs on its own CUDA stream, the most expensive first (cost per particle
~ P_max * sum_j (L_j + 1)^3, the Wigner terms of the refinement), which lets
the smaller groups fill the GPU while the largest one runs.
"""


def group_cost(n_particles: int, P_max: int, L_sched) -> float:
    """Relative refinement cost of a group: particles x P x sum_j (L_j+1)^3."""
    return float(n_particles) * P_max * sum((L + 1) ** 3 for L in L_sched)


def launch_order(costs):
    """Indices of the groups in decreasing cost (ties keep the given order)."""
    return sorted(range(len(costs)), key=lambda i: -costs[i])


def align_groups(groups):
    """Align every group; returns one output dict per group, in the given order.

    groups: list of dicts with keys ``plan``, ``particles``, ``templates`` and
    optionally ``P_per`` (int32 [B]), ``ws`` (workspace) and ``out``.
    """
    import torch
    from . import matcha_align
    costs = [group_cost(g["particles"].shape[0], g["plan"].P, g["plan"].L_sched) for g in groups]
    caller = torch.cuda.current_stream()
    results = [None] * len(groups)
    streams = []
    for i in launch_order(costs):
        g = groups[i]
        s = torch.cuda.Stream()
        s.wait_stream(caller)  # inputs produced on the caller's stream
        with torch.cuda.stream(s):
            results[i] = matcha_align(g["plan"], g["particles"], g["templates"],
                                      P_per=g.get("P_per"), ws=g.get("ws"), out=g.get("out"))
        streams.append(s)
    for s in streams:
        caller.wait_stream(s)
    return results
