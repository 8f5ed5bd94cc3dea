"""Oracle for the learned timestep proposal (test infrastructure only).

The paper has no learned component; this follows the library's stated
definitions, restated here plainly so the CUDA kernels can be checked:

Features (64 per state, FP32), at an accepted state with production F+,
depletion rate k and the previous accepted step dt_prev:
  f0 = ln T9, f1 = ln rho, f2 = ln dt_prev,
  f3 = fraction of species with k_i dt_prev >= kappa (the asymptotic branch, Sec. 3),
  f4..f23, f24..f43, f44..f63 = 20 quantiles (probabilities (m + 0.5)/20) of the
  FP32 values Y_i, F+_i and F-_i = k_i Y_i over species, read from a 64-bin
  histogram of their binary exponents: bin = clamp((e + 100) >> 2, 0, 63)
  with e the FP32 exponent (values below 2^-100, and zero, fall in bin 0), the
  quantile linearly interpolated inside its bin, expressed in log10 units.
Label: ln(dt*/dt_prev), dt* the largest step of the grid dt_prev * 2^(q/4),
  q = -8, -7, ..., 16 (clipped to t_end - t), below the first grid step whose
  kappa-switched update fails the accept test from the state; -2 ln 2 if the
  smallest fails.  (Acceptance is not monotone in dt where the asymptotic
  update flip-flops, so the largest passing step overall can sit above a
  failing one; the first failure is what a proposal can learn.)
MLP: 64 -> 128 (ReLU) -> 128 (ReLU) -> 1 on normalised features
  x = (f - mu) / sigma.  Loss: mean squared error.  Adam (Kingma & Ba 2015).

Everything here is FP64 numpy except the feature binning, which is defined on
FP32 values; matmuls are library primitives used as single steps.
"""
from __future__ import annotations

import math

import numpy as np

N_FEAT = 64
HIDDEN = 128
N_Q = 20
N_BINS = 64
GRID_HI, GRID_LO = 16, -8


# --------------------------------------------------------------------------
# features
# --------------------------------------------------------------------------
def exponent_bins(x32: np.ndarray) -> np.ndarray:
    """Histogram bin of each FP32 value from its exponent bits."""
    b = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32)
    e = ((b >> 23) & 0xFF).astype(np.int64) - 127
    e = np.where((b & 0x7FFFFFFF) == 0, -1000, e)       # zero
    e = np.where(((b >> 23) & 0xFF) == 0, -1000, e)     # subnormal: below 2^-100 anyway
    return np.clip((e + 100) >> 2, 0, N_BINS - 1)


def quantiles_from_hist(counts: np.ndarray, n: int) -> np.ndarray:
    """20 quantiles (log10 units) from a 64-bin exponent histogram of n values."""
    out = np.empty(N_Q, dtype=np.float32)
    for m in range(N_Q):
        target = np.float32((m + 0.5) / N_Q) * np.float32(n)
        cum = 0
        q = np.float32(N_BINS)
        for b in range(N_BINS):
            c = int(counts[b])
            if c > 0 and cum + c > target:
                q = np.float32(b) + (target - np.float32(cum)) / np.float32(c)
                break
            cum += c
        out[m] = (q * np.float32(4.0) - np.float32(100.0)) * np.float32(0.30102999566398120)
    return out


def features(lnT9: float, lnrho: float, dt_prev: float, Y, Fp, kk, kappa: float = 1.0) -> np.ndarray:
    Y = np.asarray(Y, dtype=np.float64)
    Fp = np.asarray(Fp, dtype=np.float64)
    kk = np.asarray(kk, dtype=np.float64)
    N = Y.shape[0]
    f = np.empty(N_FEAT, dtype=np.float32)
    f[0] = np.float32(lnT9)
    f[1] = np.float32(lnrho)
    f[2] = np.float32(math.log(dt_prev))
    f[3] = np.float32(np.count_nonzero(kk * dt_prev >= kappa)) / np.float32(N)
    y32 = Y.astype(np.float32)
    quantities = (y32, Fp.astype(np.float32), kk.astype(np.float32) * y32)
    for q, x in enumerate(quantities):
        counts = np.bincount(exponent_bins(x), minlength=N_BINS)
        f[4 + N_Q * q: 4 + N_Q * (q + 1)] = quantiles_from_hist(counts, N)
    return f


def label(orc, Y, Fp, kk, dt_prev: float, t: float, t_end: float, opts=None) -> float:
    """ln(dt*/dt_prev): walk the grid up from the smallest step and stop at
    the first failure (or at t_end)."""
    best = -2.0 * math.log(2.0)
    for q in range(GRID_LO, GRID_HI + 1):
        h = dt_prev * 2.0 ** (q / 4.0)
        h = min(h, t_end - t)
        Yn, _ = orc.update(Y, Fp, kk, h)
        if not orc.test(Y, Yn, opts)[0]:
            break
        best = math.log(h / dt_prev)
        if h >= t_end - t:
            break
    return best


# --------------------------------------------------------------------------
# MLP
# --------------------------------------------------------------------------
def init_params(seed: int = 0):
    """He-uniform weights, zero biases (FP64)."""
    rng = np.random.default_rng(seed)
    def he(fan_in, shape):
        lim = math.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, shape)
    return {"W1": he(N_FEAT, (N_FEAT, HIDDEN)), "b1": np.zeros(HIDDEN),
            "W2": he(HIDDEN, (HIDDEN, HIDDEN)), "b2": np.zeros(HIDDEN),
            "W3": he(HIDDEN, (HIDDEN, 1)), "b3": np.zeros(1)}


def forward(p, X):
    """X [B, 64] (already normalised) -> out [B], plus the activations."""
    z1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    out = (h2 @ p["W3"] + p["b3"])[:, 0]
    return out, (X, z1, h1, z2, h2)


def loss(p, X, y):
    out, _ = forward(p, X)
    return float(np.mean((out - y) ** 2))


def backward(p, X, y):
    """Gradients of the mean squared error w.r.t. every parameter."""
    out, (X, z1, h1, z2, h2) = forward(p, X)
    B = X.shape[0]
    dout = (2.0 / B) * (out - y)[:, None]
    g = {"W3": h2.T @ dout, "b3": dout.sum(0)}
    dh2 = dout @ p["W3"].T
    dz2 = dh2 * (z2 > 0)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ p["W2"].T
    dz1 = dh1 * (z1 > 0)
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(0)
    return g


def adam_step(p, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (in place) with bias correction."""
    for k in p:
        m[k] = b1 * m[k] + (1 - b1) * g[k]
        v[k] = b2 * v[k] + (1 - b2) * g[k] ** 2
        mh = m[k] / (1 - b1 ** step)
        vh = v[k] / (1 - b2 ** step)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
