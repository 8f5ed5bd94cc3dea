"""Seeded synthetic inputs (networks and zone conditions).

The only module that both the CPU oracle and the CUDA path draw from.  It
holds no integration arithmetic: rates, fluxes, updates and the timestep
controller live in the library and, separately, in the oracle.
"""
from .networks import (SWEEP_SIZES, Network, binding_energies, chain_network, custom_network, general_network,
                       net150, net365, pair_network, random_tiny_network, sweep_network)
from .rng import SplitMix64
from .zones import (UNEVEN_T_END, Zones, constant_zones, mixed_assignment, profile_zones, uneven_batch, T_START,
                    T_END)

__all__ = [
    "Network", "binding_energies", "chain_network", "custom_network", "general_network", "net150", "net365",
    "pair_network", "random_tiny_network", "sweep_network", "SWEEP_SIZES", "SplitMix64", "Zones", "constant_zones",
    "profile_zones", "mixed_assignment", "uneven_batch", "UNEVEN_T_END", "T_START", "T_END",
]
