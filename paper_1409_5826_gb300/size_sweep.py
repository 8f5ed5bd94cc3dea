"""Scaling with network size: the time of one integration step for a single
network against its number of species (the paper's single-network study:
one zone at constant T = 7e9 K and rho = 1e8 g/cm^3, Type Ia conditions),
plus the batch throughput of the same network at each size.

Only the GPU side lives here; it runs entirely in the library's kernels.  The
CPU legs of the comparison (the oracle's explicit step and dense-LU backward
Euler) are timed by bench.py --sweep.
"""
from __future__ import annotations

import time

import numpy as np

from kn_inputs import SWEEP_SIZES, constant_zones, profile_zones, sweep_network

from . import kn

T9 = 7.0
RHO = 1e8
T_END = 1e-3  # long enough that every run ends at its step limit


def single_zone_step_time(net, steps: int = 2000, precision: int = kn.PREC_MIXED, stream=None,
                          T9: float = T9, rho: float = RHO) -> dict:
    """One zone at constant (T9, rho), `steps` attempts: the fastest one-group
    tiling's time per accepted step and per attempt (CUDA events around the
    launch)."""
    import torch
    zones = constant_zones(net, 1, T9=T9, rho=rho, t_end=T_END)
    g = kn.Network(net)
    n = int(net.n_species)
    cands = sorted({min(1024, max(64, (n + 31) // 32 * 32)), 128, 256, 512, 1024})
    best = None
    for G in cands:
        o = kn.Opts(precision=precision, max_steps=steps, threads_per_zone=G, threads_per_cta=G, use_graph=1)
        try:
            g.set_zones(zones, stream)
            kn.integrate_batch([g], o, stream)  # warm-up (tables, graph)
            ms = []
            for _ in range(3):
                g.set_zones(zones, stream)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                kn.integrate_batch([g], o, stream)
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
        except kn.KnError:
            continue  # this group size does not fit the network
        r = g.get(stream)
        acc, att = int(r["steps"][0]), int(r["steps"][0] + r["rejects"][0])
        t = float(np.median(ms)) / 1e3
        cur = {"threads_per_zone": G, "s_per_step": t / max(1, acc), "s_per_attempt": t / max(1, att),
               "steps": acc, "attempts": att, "status": int(r["status"][0])}
        if best is None or cur["s_per_step"] < best["s_per_step"]:
            best = cur
    g.close()
    return best


def batch_throughput(net, n_zones: int = 4096, t_end: float = 1e-10, precision: int = kn.PREC_MIXED,
                     stream=None) -> dict:
    """Autotuned batch of profiled zones: accepted zone-steps/s of one launch."""
    import torch
    zones = profile_zones(net, n_zones, t_end=t_end)
    g = kn.Network(net)
    g.set_zones(zones, stream)
    tiling = kn.autotune([g], kn.Opts(precision=precision), max_steps=200, stream=stream)
    o = kn.Opts(precision=precision, use_graph=1)
    g.set_zones(zones, stream)
    kn.integrate_batch([g], o, stream)
    torch.cuda.synchronize()
    g.set_zones(zones, stream)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    kn.integrate_batch([g], o, stream)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    st = kn.batch_stats([g], stream)
    g.close()
    return {"zones": n_zones, "zone_steps_per_s": st["steps"] / t, "zones_ok": st["zones_ok"],
            "tiling": {"threads_per_zone": tiling.get("threads_per_zone"),
                       "threads_per_cta": tiling.get("threads_per_cta")}}


def run(sizes=SWEEP_SIZES, steps: int = 2000, batch_zones: int = 4096, stream=None) -> list[dict]:
    """The GPU side of the sweep, one row per network size."""
    rows = []
    for n in sizes:
        net = sweep_network(n)
        t0 = time.perf_counter()
        row = {"n_species": int(net.n_species), "n_reactions": int(net.n_reactions), "network": net.name}
        row["gpu_single_zone"] = single_zone_step_time(net, steps, stream=stream)
        row["gpu_batch"] = batch_throughput(net, batch_zones, stream=stream)
        row["wall_s"] = time.perf_counter() - t0
        rows.append(row)
    return rows
