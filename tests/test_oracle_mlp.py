"""Pins of the learned-timestep oracle (oracle/mlp.py): gradients against
central finite differences, the forward pass against its affine collapse in
the all-active regime, Adam's first-step property, the exponent binning
against frexp, and quantiles against closed forms."""
import math

import numpy as np
import pytest

import oracle.mlp as M


def _params(seed=1, scale=1.0):
    p = M.init_params(seed)
    rng = np.random.default_rng(seed + 7)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.1, p[k].shape)
    return {k: v * scale if k.startswith("W") else v for k, v in p.items()}


def test_gradients_match_central_differences():
    rng = np.random.default_rng(0)
    p = _params()
    X = rng.normal(size=(9, M.N_FEAT))
    y = rng.normal(size=9)
    g = M.backward(p, X, y)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = M.loss(p, X, y)
            flat[i] = old - h
            lm = M.loss(p, X, y)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, i, fd, an)


def test_forward_collapses_to_affine_map_when_all_units_active():
    # positive inputs, weights and biases keep every ReLU in its linear part,
    # so the network is x -> x W1 W2 W3 + (b1 W2 W3 + b2 W3 + b3)
    rng = np.random.default_rng(2)
    p = {"W1": rng.uniform(0.01, 0.1, (64, 128)), "b1": rng.uniform(0, 0.1, 128),
         "W2": rng.uniform(0.01, 0.1, (128, 128)), "b2": rng.uniform(0, 0.1, 128),
         "W3": rng.uniform(-0.1, 0.1, (128, 1)), "b3": np.array([0.3])}
    X = rng.uniform(0, 1, (5, 64))
    out, acts = M.forward(p, X)
    assert (acts[1] > 0).all() and (acts[3] > 0).all()
    Wc = p["W1"] @ p["W2"] @ p["W3"]
    bc = p["b1"] @ p["W2"] @ p["W3"] + p["b2"] @ p["W3"] + p["b3"]
    assert np.allclose(out, (X @ Wc)[:, 0] + bc, rtol=1e-12)
    # and a negative pre-activation contributes nothing (ReLU kink)
    p["b1"][:] = -1e6
    out, _ = M.forward(p, X)
    assert np.allclose(out, (np.maximum(p["b2"], 0) @ p["W3"])[0] + p["b3"][0])


def test_adam_first_step_moves_by_lr_times_sign():
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([3e-3, -7.0, 1e4])}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    M.adam_step(p, g, m, v, step=1, lr=0.01, eps=0.0)
    assert np.allclose(p["w"], [1.0 - 0.01, -2.0 + 0.01, 0.5 - 0.01], rtol=0, atol=1e-15)


def test_adam_converges_on_quadratic():
    target = np.array([0.5, -1.5, 2.0])
    p = {"w": np.zeros(3)}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    for s in range(1, 3001):
        M.adam_step(p, {"w": p["w"] - target}, m, v, step=s, lr=0.01)
    assert np.allclose(p["w"], target, atol=1e-3)


def test_exponent_bins_match_frexp():
    rng = np.random.default_rng(4)
    x = (10.0 ** rng.uniform(-45, 38, 2000)).astype(np.float32)
    x[:5] = [0.0, 1.0, 2.0 ** -100, 2.0 ** -101, 3.0e38]
    b = M.exponent_bins(x)
    for xi, bi in zip(x, b):
        if xi == 0 or xi < 2.0 ** -126:
            assert bi == 0
            continue
        m, e = math.frexp(float(xi))  # xi = m 2^e, m in [0.5, 1): floor(log2 xi) = e - 1
        assert bi == min(max((e - 1 + 100) >> 2, 0), 63)


def test_quantiles_closed_forms():
    # n equal values 1.0: exponent 0 -> bin 25; quantile p sits at 25 + p,
    # i.e. log2 value 4 (25 + p) - 100 = 4 p
    n = 40
    counts = np.bincount(M.exponent_bins(np.ones(n, np.float32)), minlength=64)
    q = M.quantiles_from_hist(counts, n)
    p = (np.arange(20) + 0.5) / 20
    assert np.allclose(q, 4 * p * math.log10(2), rtol=1e-6, atol=1e-5)  # FP32 cancellation in 4q - 100
    # one value in each of the bins 10..29: quantile m falls in bin 10 + m at 0.5
    vals = np.array([2.0 ** (4 * b - 100) for b in range(10, 30)], np.float32)
    counts = np.bincount(M.exponent_bins(vals), minlength=64)
    q = M.quantiles_from_hist(counts, 20)
    assert np.allclose(q, (4 * (10 + np.arange(20) + 0.5) - 100) * math.log10(2), rtol=1e-6)


def test_features_layout_and_label_property(oracle_mod):
    from kn_inputs import constant_zones, net150
    net = net150()
    orc = oracle_mod.Oracle(net)
    z = constant_zones(net, t_end=1e-9)
    r = orc.integrate(z, 0, record=300)
    Y, t = orc.replay(z, 0, r["dts"][:200])
    dt_prev = r["dts"][199]
    k = orc.rates(3.0, 1e8)
    Fp, kk, _ = orc.rhs(k, Y)
    f = M.features(math.log(3.0), math.log(1e8), dt_prev, Y, Fp, kk)
    assert f.shape == (64,) and f.dtype == np.float32
    assert f[0] == np.float32(math.log(3.0)) and f[2] == np.float32(math.log(dt_prev))
    assert 0 <= f[3] <= 1
    for q in range(3):
        assert np.all(np.diff(f[4 + 20 * q: 24 + 20 * q]) >= 0)  # quantiles are monotone
    lab = M.label(orc, Y, Fp, kk, dt_prev, t, z.t_end[0])
    q = round(lab / math.log(2) * 4)
    for qq in range(M.GRID_LO, q + 1):              # every grid step up to the label passes ...
        Yn, _ = orc.update(Y, Fp, kk, dt_prev * 2 ** (qq / 4))
        assert orc.test(Y, Yn)[0]
    if q < M.GRID_HI:                               # ... and the next one up fails
        Yn, _ = orc.update(Y, Fp, kk, dt_prev * 2 ** ((q + 1) / 4))
        assert not orc.test(Y, Yn)[0]
