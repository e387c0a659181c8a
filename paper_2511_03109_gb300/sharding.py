"""theta-sharding across GPUs: each rank owns a replica of the parametric matrix and its own
share of the thetas; the only cross-rank traffic is a barrier and a max-reduction of timers.

The online stage for one theta is independent of every other theta (§4.4), so a batch of
thetas partitions across ranks with no exchange on the data path.
"""
from __future__ import annotations


def shard(items, rank: int, world: int):
    """Round-robin share of `items` owned by `rank` (ranks 0..world-1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    return items[rank::world]


def owner(index: int, world: int) -> int:
    """Rank that owns item `index` under `shard`."""
    return index % world


def max_over_ranks(value: float, dist=None) -> float:
    """Max of a per-rank scalar (a step time) over the process group; identity without one."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
