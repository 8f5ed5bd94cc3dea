"""Operator-split driver (Sec. 4, Sec. 6): the network advances every zone
over one hydro interval at a time, with T and rho held constant over the
interval, abundances and the final dt carried into the next one, and the
host's own work (the hydro step) running while the GPU integrates (Sec. 5:
launch asynchronously, then do the CPU work).
"""
from __future__ import annotations

import numpy as np

from . import kn


def run(net_gpu: "kn.Network", zones, schedule, opts: "kn.Opts", host_step=None, stream=None):
    """Integrate `zones` (kn_inputs.Zones, host) through the hydro intervals of
    `schedule`: a list of (T9 [Z], rho [Z], t_end [Z]) per interval; the first
    interval starts from `zones` (its T0, rho0 are replaced by the first
    entry's).  `host_step(k)` runs on the host while interval k integrates.
    Returns per interval the host copy of the results plus the energy release."""
    z0 = zones
    T9, rho, te = schedule[0]
    first = type(z0)(Y0=z0.Y0, T0=np.asarray(T9, float), rho0=np.asarray(rho, float), tau=np.zeros(z0.n_zones),
                     t_start=z0.t_start, t_end=np.asarray(te, float), dt_trial=z0.dt_trial)
    net_gpu.set_zones(first, stream)
    out = []
    for k, (T9, rho, te) in enumerate(schedule):
        if k > 0:
            net_gpu.advance(T9, rho, te, stream)
        kn.integrate_batch([net_gpu], opts, stream)   # asynchronous
        if host_step is not None:
            host_step(k)                               # host work overlaps the integration
        r = net_gpu.get(stream)                        # synchronises
        r["energy"] = net_gpu.energy(stream)
        out.append(r)
    return out
