"""Host-side sharding of independent environments over ranks (one GPU per
rank, no collective inside a step) and the reductions of the timing
harness.

Environments never interact, so a batch is split into contiguous env ranges
(the library lays every per-env quantity out contiguously), balanced by a
per-env weight such as the tet count; each rank steps its own range.
"""


def shard_envs(weights, world):
    """Contiguous (start, end) env ranges, one per rank, covering every env
    once, with each range's weight close to total / world (a range ends at
    the first env whose cumulative weight reaches the rank's share)."""
    n = len(weights)
    if world < 1:
        raise ValueError("world must be >= 1")
    total = float(sum(weights))
    out, start, acc = [], 0, 0.0
    for r in range(world):
        if r == world - 1:
            out.append((start, n))
            break
        target = total * (r + 1) / world
        end = start
        while end < n and (acc + weights[end] <= target or end == start) and n - end > world - 1 - r:
            acc += weights[end]
            end += 1
        out.append((start, end))
        start = end
    return out


def max_over_ranks(x, dist=None, device="cpu"):
    """x reduced with max over the ranks of the default process group (x
    itself without one): the job's time is its slowest rank's."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
