"""Zone sharding across GPUs (one process per GPU, no collective in the data
path): zones are independent networks (Sec. 9), so rank r integrates its own
slice of the global batch and the ranks only exchange the timing scalars.
"""
from __future__ import annotations


def zone_slice(rank: int, world: int, zones_per_rank: int) -> tuple[int, int]:
    """Global zone indices [lo, hi) of `rank` (weak scaling: a fixed count per rank)."""
    if not (0 <= rank < world) or zones_per_rank < 1:
        raise ValueError("bad rank / world / zones_per_rank")
    lo = rank * zones_per_rank
    return lo, lo + zones_per_rank


def zone_seed_base(rank: int, world: int, zones_per_rank: int, base_seed: int = 1000) -> int:
    """Seed of the rank's first zone, so the shards tile the global batch
    seeded base_seed + global zone index."""
    return base_seed + zone_slice(rank, world, zones_per_rank)[0]


def aggregate(ms: float, steps: int, zones_ok: int, device=None) -> tuple[float, int, int]:
    """Max elapsed time and summed work over the ranks (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), int(steps), int(zones_ok)
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([steps, zones_ok], dtype=torch.float64, device=device)
    dist.all_reduce(c)
    return float(t.item()), int(c[0].item()), int(c[1].item())
