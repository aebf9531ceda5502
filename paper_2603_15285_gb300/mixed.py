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


class MixedBatch:
    """A mixed batch bound to fixed device buffers.

    Each group gets its workspace and outputs once; with ``autotune`` each
    group's plan is tuned on its own data first (``Plan.autotune``: tile
    choices that change no result bit).  ``run()`` launches the groups
    eagerly (concurrent streams, costliest first); ``capture()`` records that
    launch sequence, fork and join included, into one CUDA graph that
    ``replay()`` relaunches on the current stream.
    """

    def __init__(self, groups, autotune: bool = True):
        import torch
        from . import alloc_workspace
        self.groups = []
        self.tune = []
        for g in groups:
            plan, parts = g["plan"], g["particles"]
            B = parts.shape[0]
            d = dict(g)
            d["ws"] = alloc_workspace(plan, B)
            dev = parts.device
            d["out"] = dict(euler=torch.empty((B, 3), dtype=torch.float64, device=dev),
                            R=torch.empty((B, 3, 3), dtype=torch.float64, device=dev),
                            score=torch.empty((B,), dtype=torch.float64, device=dev),
                            best_p=torch.empty((B,), dtype=torch.int32, device=dev),
                            flags=torch.empty((B,), dtype=torch.int32, device=dev))
            self.tune.append(plan.autotune(parts, g["templates"], ws=d["ws"], P_per=g.get("P_per"))
                             if autotune else None)
            self.groups.append(d)
        self.graph = None

    @property
    def outputs(self):
        return [g["out"] for g in self.groups]

    def run(self):
        return align_groups(self.groups)

    def capture(self):
        import torch
        self.run()  # first calls on every plan happen outside the capture
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        cs = torch.cuda.Stream()
        cs.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(cs):
            with torch.cuda.graph(graph, stream=cs):
                align_groups(self.groups)
        torch.cuda.current_stream().wait_stream(cs)
        self.graph = graph
        return self

    def replay(self):
        self.graph.replay()
        return self.outputs
