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
                  stream=None):
    """Train a fresh network on the records with the library's GPU kernels
    (mean squared error, Adam).  Returns (network, per-epoch mean loss)."""
    import torch
    mu, sd = normalisation(feat)
    net = kn.MLP()
    net.set_params(init_params(seed), mu, sd)
    n = feat.shape[0]
    gen = torch.Generator(device=feat.device)
    gen.manual_seed(seed)
    loss = torch.zeros(1, dtype=torch.float32, device=feat.device)
    history = []
    for _ in range(epochs):
        perm = torch.randperm(n, device=feat.device, generator=gen)
        tot, cnt = 0.0, 0
        for i in range(0, n - batch + 1, batch):
            idx = perm[i:i + batch]
            xb = feat.index_select(0, idx).contiguous()
            yb = lab.index_select(0, idx).contiguous()
            net.backward(xb, yb, loss, stream)
            net.adam(lr, stream=stream)
            tot += float(loss.item()) if (cnt % 64 == 0) else 0.0
            cnt += 1
        history.append(tot / max(1, (cnt + 63) // 64))
    return net, history
