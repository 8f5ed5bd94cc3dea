"""Seeded per-zone conditions: initial abundances and the T9(t), rho(t) profile.

A zone is one hydro cell's network problem (Sec. 6: abundances, temperature,
density, the hydro interval and a trial timestep are what the host sends).
The profile is T9(t) = T0 exp(-t/tau), rho(t) = rho0 exp(-3 t/tau); tau <= 0
means T9 = T0 and rho = rho0 held constant (the operator-split setting of
Sec. 4).  Zone z of a batch draws from SplitMix64(base_seed + z).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .networks import Network
from .rng import SplitMix64

T_START = 1e-12
T_END = 1e-2


@dataclass
class Zones:
    Y0: np.ndarray        # [Z, N] molar abundances, sum_i A_i Y_i = 1
    T0: np.ndarray        # [Z] T9 at t = 0
    rho0: np.ndarray      # [Z] g/cm^3 at t = 0
    tau: np.ndarray       # [Z] profile e-folding time (s); <= 0 means constant
    t_start: np.ndarray   # [Z]
    t_end: np.ndarray     # [Z]
    dt_trial: np.ndarray  # [Z] first trial network timestep

    @property
    def n_zones(self) -> int:
        return int(self.T0.shape[0])

    def subset(self, idx) -> "Zones":
        idx = np.asarray(idx)
        return Zones(*(getattr(self, f)[idx].copy() for f in
                       ("Y0", "T0", "rho0", "tau", "t_start", "t_end", "dt_trial")))


def constant_zones(net: Network, n_zones: int = 1, T9: float = 3.0, rho: float = 1e8,
                   t_start: float = T_START, t_end: float = T_END,
                   dt_trial: float | None = None, Y0=None) -> Zones:
    """n identical zones at constant T9, rho."""
    y = net.initial_Y() if Y0 is None else np.asarray(Y0, dtype=np.float64)
    z = n_zones
    return Zones(
        Y0=np.tile(y, (z, 1)),
        T0=np.full(z, float(T9)),
        rho0=np.full(z, float(rho)),
        tau=np.zeros(z),
        t_start=np.full(z, float(t_start)),
        t_end=np.full(z, float(t_end)),
        dt_trial=np.full(z, float(t_start if dt_trial is None else dt_trial)),
    )


def profile_zones(net: Network, n_zones: int, base_seed: int = 1000,
                  t_start: float = T_START, t_end: float = T_END) -> Zones:
    """Batched zones with T0 ~ U[2, 7], rho0 ~ logU[1e7, 1e9], tau ~ logU[0.1, 1] s."""
    y = net.initial_Y()
    T0 = np.empty(n_zones)
    rho0 = np.empty(n_zones)
    tau = np.empty(n_zones)
    for z in range(n_zones):
        rng = SplitMix64(base_seed + z)
        T0[z] = 2.0 + 5.0 * rng.uniform()
        rho0[z] = math.exp(math.log(1e7) + rng.uniform() * (math.log(1e9) - math.log(1e7)))
        tau[z] = math.exp(math.log(0.1) + rng.uniform() * (math.log(1.0) - math.log(0.1)))
    return Zones(
        Y0=np.tile(y, (n_zones, 1)),
        T0=T0, rho0=rho0, tau=tau,
        t_start=np.full(n_zones, float(t_start)),
        t_end=np.full(n_zones, float(t_end)),
        dt_trial=np.full(n_zones, float(t_start)),
    )


def mixed_assignment(n_zones: int = 2048, ratio=(1, 2, 1), seed: int = 7) -> np.ndarray:
    """Network index (0, 1, 2) of each zone for a mixed-size batch, shuffled."""
    tot = sum(ratio)
    counts = [n_zones * r // tot for r in ratio]
    counts[1] += n_zones - sum(counts)
    lab = []
    for k, c in enumerate(counts):
        lab += [k] * c
    SplitMix64(seed).shuffle(lab)
    return np.asarray(lab, dtype=np.int32)


# The uneven-size batch: the chain over its own interval (1e-12 -> 1e-2 s), the
# 150- and 365-species networks over 1e-12 -> 1e-9 s.
UNEVEN_T_END = {"chain16_48": 1e-2, "net150_1604": 1e-9, "net365_4400": 1e-9}


def uneven_batch(n_zones: int = 2048, ratio=(1, 2, 1), seed: int = 7):
    """The uneven-size batch: n_zones zones of the 16/48, 150/1604 and
    365/4400 networks in `ratio`, shuffled (mixed_assignment); zone z of the
    batch draws its profile from seed 1000 + z whatever its network.
    Returns [(name, network, zones, batch indices)] in network order."""
    from .networks import chain_network, net150, net365
    lab = mixed_assignment(n_zones, ratio, seed)
    out = []
    for k, (name, net) in enumerate((("chain16_48", chain_network()), ("net150_1604", net150()),
                                     ("net365_4400", net365()))):
        idx = np.nonzero(lab == k)[0]
        z = profile_zones(net, n_zones, t_end=UNEVEN_T_END[name]).subset(idx)
        out.append((name, net, z, idx))
    return out
