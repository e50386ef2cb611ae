"""Placement of independent problems on ranks (one process per GPU).

Independent problems share nothing on the data path, so a multi-GPU run of
a batch gives every rank a subset and needs no collective except the
max-over-ranks time of the benchmark.  `partition` balances an estimate of
each problem's work (greedy longest-first onto the least-loaded rank); it is
deterministic, so every rank computes the same placement without talking.
"""


def work_estimate(spec, N=8):
    """Relative cost of one RK4 step of a problem from `inputs.batched_problems`:
    elements x per-element cost (an element PCG stage costs about 40x a
    modal-route element stage at N = 8)."""
    elements = spec["n"] * spec["n"]
    per_element = 40.0 if spec.get("variable") else 1.0
    return elements * per_element * (N + 1) ** 2 / 81.0


def partition(specs, world, cost=work_estimate):
    """List of `world` lists of problem indices: disjoint, covering, each
    sorted; greedy longest-processing-time-first (ties by index)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(specs)), key=lambda i: (-cost(specs[i]), i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += cost(specs[i])
    return [sorted(x) for x in out]


def max_over_ranks(value):
    """Maximum of a float over the ranks of the default process group (the
    value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
