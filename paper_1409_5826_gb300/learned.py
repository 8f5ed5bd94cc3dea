"""Learned timestep proposal: data generation, training and deployment helpers.

The integrator itself generates the training data (kn_opts.record_*): at every
state reached by an accepted step it writes the 64 features and the label
ln(dt_best/dt_prev), dt_best the largest grid step dt_prev 2^(q/4) that passes
the accept test from that state.  The network is trained on the GPU by the
library's BF16 kernels (kn_mlp_backward / kn_mlp_adam) and deployed through
kn_opts.mlp, where the plain controller stays the judge of every step.
"""
from __future__ import annotations

import numpy as np

from . import kn

N_FEAT = 64


def generate_records(jobs, capacity: int, precision: int = kn.PREC_MIXED, stream=None):
    """Run the integrator in record mode over (network, zones) jobs until
    `capacity` records are collected.  Returns (features [n, 64] float32,
    labels [n] float32) as torch CUDA tensors."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    feat = torch.empty((capacity, N_FEAT), dtype=torch.float32, device=dev)
    lab = torch.empty(capacity, dtype=torch.float32, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    for net, zones in jobs:
        g = kn.Network(net)
        g.set_zones(zones, stream)
        o = kn.Opts(precision=precision, record_features=feat.data_ptr(), record_labels=lab.data_ptr(),
                    record_capacity=capacity, record_count=count.data_ptr())
        kn.integrate_batch([g], o, stream)
        torch.cuda.synchronize()
        g.close()
        if int(count.item()) >= capacity:
            break
    n = min(int(count.item()), capacity)
    return feat[:n], lab[:n]


def normalisation(feat) -> tuple[np.ndarray, np.ndarray]:
    """Per-feature mean and standard deviation (floor 1e-3) of the records."""
    f = feat.double()
    mu = f.mean(0).cpu().numpy().astype(np.float32)
    sd = f.std(0).clamp_min(1e-3).cpu().numpy().astype(np.float32)
    return mu, sd


def _he_uniform(rng, fan_in, shape):
    lim = np.sqrt(6.0 / fan_in)
    return rng.uniform(-lim, lim, shape)


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases, flattened in the kn.h parameter order."""
    rng = np.random.default_rng(seed)
    p = {"W1": _he_uniform(rng, N_FEAT, (N_FEAT, 128)), "b1": np.zeros(128),
         "W2": _he_uniform(rng, 128, (128, 128)), "b2": np.zeros(128),
         "W3": _he_uniform(rng, 128, (128, 1)), "b3": np.zeros(1)}
    return kn.mlp_pack(p)


def train_network(feat, lab, epochs: int = 4, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
                  stream=None, time_kernels: bool = False):
    """Train a fresh network on the records with the library's GPU kernels
    (mean squared error, Adam).  Each epoch shuffles the records once on the
    GPU; batches are then contiguous slices.  Returns (network, per-epoch
    mean loss), plus with time_kernels the seconds the training kernels
    themselves took (CUDA events around each batch's backward and Adam)."""
    import torch
    mu, sd = normalisation(feat)
    net = kn.MLP()
    net.set_params(init_params(seed), mu, sd)
    n = feat.shape[0]
    gen = torch.Generator(device=feat.device)
    gen.manual_seed(seed)
    losses = torch.zeros(max(1, n // batch), dtype=torch.float32, device=feat.device)
    history = []
    events = []
    st = stream if stream is not None else torch.cuda.current_stream()
    for _ in range(epochs):
        perm = torch.randperm(n, device=feat.device, generator=gen)
        xs = feat.index_select(0, perm)
        ys = lab.index_select(0, perm)
        nb = 0
        for i in range(0, n - batch + 1, batch):
            if time_kernels:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
            net.backward(xs[i:i + batch], ys[i:i + batch], losses[nb:nb + 1], stream)
            net.adam(lr, stream=stream)
            if time_kernels:
                e1.record(st)
                events.append((e0, e1))
            nb += 1
        history.append(float(losses[:nb].mean().item()))
    if time_kernels:
        torch.cuda.synchronize()
        return net, history, sum(a.elapsed_time(b) for a, b in events) / 1e3
    return net, history
