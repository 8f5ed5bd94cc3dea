"""Zone sharding across GPUs (one process per GPU, no collective in the data
path): zones are independent networks (Sec. 9), so rank r integrates its own
slice of the global batch and the ranks only exchange the timing scalars.

Two partitions: weak scaling gives every rank its own fixed-size slice of a
global batch seeded by zone index; strong scaling splits one fixed batch over
the ranks balanced by predicted cost.
"""
from __future__ import annotations

import numpy as np


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


def cost_key(net, zones) -> np.ndarray:
    """Per-zone ordering key of predicted integration cost: the mean log-rate
    at the zone's initial conditions, nbar ln T0 + rbar ln rho0 (nbar the mean
    temperature exponent, rbar the mean reactant count less one); stiffer zones
    take more steps.  The same key orders the integrator's work queue."""
    nbar = float(np.mean(net.t9_exp))
    rbar = float(np.mean(np.asarray(net.n_reac, dtype=np.float64) - 1.0))
    return nbar * np.log(np.asarray(zones.T0, np.float64)) + rbar * np.log(np.asarray(zones.rho0, np.float64))


def balanced_partition(keys, world: int) -> list:
    """Zone indices of each rank for a strong-scaling split of one batch:
    zones in descending key order are dealt to the ranks in a serpentine
    order (0, 1, ..., W-1, W-1, ..., 0, 0, 1, ...), so every rank gets an
    equal share of each cost quantile whatever the cost's magnitude as a
    function of the key.  Rank sizes differ by at most one zone."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = np.argsort(-np.asarray(keys, np.float64), kind="stable")
    parts = [[] for _ in range(world)]
    for pos, z in enumerate(order):
        rnd, k = divmod(pos, world)
        parts[k if rnd % 2 == 0 else world - 1 - k].append(int(z))
    return [np.sort(np.asarray(p, dtype=np.int64)) for p in parts]
