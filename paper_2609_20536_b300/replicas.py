"""Replicas over several GPUs (one process per GPU).

The points of a scan are independent HOTRG runs, so the path shards with no
data-path collective: each rank takes its share of the points, runs them
through its own context, and only the per-point scalars (ln Z/N, the step
records) are gathered on the host at the end.

``shard`` balances the shares longest-processing-time first, with the cost
model of the library's batch scheduler (the s2 work of every step plus a
fixed per-step cost), so ranks with D_cut = 64 points and ranks with
D_cut = 24 points finish together.  ``gather`` collects per-rank results with
one host-side ``all_gather_object`` (any process group: gloo, or NCCL).
"""

import heapq


def step_sizes(n_max, d_cut, n_steps, d0=None):
    """(D_h, D_v) of every step of a run from D0 = 2 n_max + 1."""
    h = v = d0 if d0 is not None else 2 * n_max + 1
    out = []
    for _ in range(n_steps):
        out.append((h, v))
        h, v = v, min(d_cut, h * h)
    return out


def point_cost(n_max, d_cut, n_steps):
    """Relative cost of one point: sum over steps of D' D_h^3 D_v^3 + 1e6."""
    c = 0.0
    for h, v in step_sizes(n_max, d_cut, n_steps):
        c += min(d_cut, h * h) * float(h) ** 3 * float(v) ** 3 + 1e6
    return c


def shard(points, world, rank):
    """Indices (ascending) of the points rank `rank` of `world` runs.

    points: sequence of objects with n_max, d_cut, n_steps.  Longest first,
    each to the least-loaded rank (ties to the lower rank), deterministic, so
    every rank computes the same partition without communicating.
    """
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need world >= 1 and 0 <= rank < world")
    costs = [point_cost(p.n_max, p.d_cut, p.n_steps) for p in points]
    order = sorted(range(len(points)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    mine = []
    for i in order:
        load, r = heapq.heappop(heap)
        if r == rank:
            mine.append(i)
        heapq.heappush(heap, (load + costs[i], r))
    return sorted(mine)


def loads(points, world):
    """Total cost per rank under ``shard`` (for reporting the balance)."""
    costs = [point_cost(p.n_max, p.d_cut, p.n_steps) for p in points]
    return [sum(costs[i] for i in shard(points, world, r)) for r in range(world)]


def gather(results, group=None):
    """Merge {point index: result} dicts of all ranks (host-side all_gather_object)."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return dict(results)
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, dict(results), group=group)
    merged = {}
    for part in parts:
        for k, v in part.items():
            if k in merged:
                raise RuntimeError(f"point {k} computed by two ranks")
            merged[k] = v
    return merged
