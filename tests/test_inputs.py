"""Seeded input generators: determinism and the structural properties the
workloads must have (sizes, A-conservation of every reaction, hub species)."""
import numpy as np
import pytest

from kn_inputs import (SplitMix64, chain_network, constant_zones, mixed_assignment, net150,
                       net365, profile_zones)


def test_splitmix64_reference_values():
    # First outputs of SplitMix64 seeded with 0 (the published algorithm's
    # well-known test vector).
    r = SplitMix64(0)
    assert r.next_u64() == 0xE220A8397B1DCDAF
    assert r.next_u64() == 0x6E789E6AA1B965F4
    assert r.next_u64() == 0x06C45D188009454F


@pytest.mark.parametrize("factory,N,R", [(chain_network, 16, 48), (net150, 150, 1604),
                                         (net365, 365, 4400)])
def test_network_shape_and_conservation(factory, N, R):
    a, b = factory(), factory()
    assert a.n_species == N and a.n_reactions == R
    for f in ("A", "reac", "prod", "ln_k0", "t9_exp"):
        assert np.array_equal(getattr(a, f), getattr(b, f))  # deterministic
    for j in range(R):
        r = a.reac[j][a.reac[j] >= 0]
        p = a.prod[j][a.prod[j] >= 0]
        assert 1 <= len(r) <= 3 and 1 <= len(p) <= 3
        assert a.A[r].sum() == a.A[p].sum()
    Y = a.initial_Y()
    assert abs(np.sum(a.A * Y) - 1.0) < 1e-15


def test_general_network_structure():
    n = net150()
    s = n.summary()
    # 1604 = 1204 base reactions (30/60/10 % 1/2/3-body) + 400 reverses
    nr = n.n_reac[:1204]
    assert [(nr == k).sum() for k in (1, 2, 3)] == [361, 723, 120]
    assert s["max_fan_in"] > 300 and s["median_fan_in"] < 40  # light hubs
    assert (n.ln_k0 >= np.log(1e-8)).all() and (n.ln_k0 <= np.log(1e10)).all()
    assert (n.t9_exp >= 0).all() and (n.t9_exp <= 8).all()
    # the last 400 reactions are reverses of base reactions
    base = {(tuple(sorted(r[r >= 0])), tuple(sorted(p[p >= 0])))
            for r, p in zip(n.reac[:1204], n.prod[:1204])}
    for r, p in zip(n.reac[1204:], n.prod[1204:]):
        assert (tuple(sorted(p[p >= 0])), tuple(sorted(r[r >= 0]))) in base


def test_zone_generators():
    n = net150()
    z = profile_zones(n, 64)
    assert z.Y0.shape == (64, 150)
    assert (z.T0 >= 2).all() and (z.T0 <= 7).all()
    assert (z.rho0 >= 1e7).all() and (z.rho0 <= 1e9).all()
    assert (z.tau >= 0.1).all() and (z.tau <= 1).all()
    z2 = profile_zones(n, 64)
    assert np.array_equal(z.T0, z2.T0) and np.array_equal(z.rho0, z2.rho0)
    c = constant_zones(n, 3, T9=3.0, rho=1e8)
    assert (c.tau == 0).all() and c.n_zones == 3
    lab = mixed_assignment(2048)
    assert np.bincount(lab).tolist() == [512, 1024, 512]


@pytest.mark.parametrize("n", [16, 32, 64, 100, 150, 250, 365])
def test_sweep_networks(n):
    from kn_inputs import SWEEP_SIZES, sweep_network
    assert n in SWEEP_SIZES
    a, b = sweep_network(n), sweep_network(n)
    assert a.n_species == n
    for f in ("A", "reac", "prod", "ln_k0", "t9_exp"):
        assert np.array_equal(getattr(a, f), getattr(b, f))  # deterministic
    for j in range(a.n_reactions):
        r = a.reac[j][a.reac[j] >= 0]
        p = a.prod[j][a.prod[j] >= 0]
        assert 1 <= len(r) <= 3 and 1 <= len(p) <= 3
        assert a.A[r].sum() == a.A[p].sum()
    # the endpoints are the benchmark networks; sizes in between interpolate
    # the reaction count between 10.69 and 12.05 per species
    if n == 150:
        assert a.n_reactions == 1604
    elif n == 365:
        assert a.n_reactions == 4400
    elif n > 16:
        assert 10.5 * n <= a.n_reactions <= 12.1 * n
    assert abs(float((a.A * a.initial_Y()).sum()) - 1.0) < 1e-12
