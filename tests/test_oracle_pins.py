"""Pins of the CPU oracle against things other than itself.

Each test ties one oracle function to what the paper or the mathematics fixes:
hand-worked values, exact rational arithmetic, closed forms, matrix powers of
linear maps, conservation laws, equilibrium fixed points, a library linear
solver, and backward Euler with Richardson extrapolation on tiny networks.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from kn_inputs import (chain_network, constant_zones, custom_network, net150, net365,
                       pair_network, profile_zones, random_tiny_network)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Sec. 3: the kappa switch and Eq. (3) on hand-worked cases
# --------------------------------------------------------------------------
def _golden_cases():
    rows = []
    for line in open(os.path.join(GOLDEN, "kappa_switch_cases.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        Y, F, k, dt, br, Yp = line.split()
        rows.append((float(Y), float(F), float(k), float(dt), br, float(Yp)))
    return rows


def test_update_hand_worked_cases(oracle_mod):
    cases = _golden_cases()
    assert len(cases) >= 8
    net = custom_network([1.0], [((0,), (0,))], [0.0], [0.0])  # one species; only update() is used
    orc = oracle_mod.Oracle(net)
    for Y, F, k, dt, br, Yp in cases:
        Yn, asy = orc.update([Y], [F], [k], dt, kappa=1.0)
        assert Yn[0] == Yp, (Y, F, k, dt, Yn[0], Yp)
        assert bool(asy[0]) == (br == "asy")


# --------------------------------------------------------------------------
# Eq. (1): fluxes, F+ and k_i against exact rational mass action
# --------------------------------------------------------------------------
def _exact_rhs(net, k, Y):
    """Mass action in exact rationals, written from multiplicities (not slots):
    F+_i = sum_j nu_prod(i,j) f_j, F-_i = sum_j nu_reac(i,j) f_j, and
    k_i = lim F-_i / Y_i = sum over reactions with nu_reac(i,j) = 1 of
    k_j prod_{other reactants} Y (+ nu Y_i^(nu-1) terms for nu > 1)."""
    N = net.n_species
    kq = [Fraction(float(x)) for x in k]
    Yq = [Fraction(float(y)) for y in Y]
    Fp = [Fraction(0)] * N
    Fm = [Fraction(0)] * N
    kk = [Fraction(0)] * N
    for j in range(net.n_reactions):
        rs = [int(s) for s in net.reac[j] if s >= 0]
        ps = [int(s) for s in net.prod[j] if s >= 0]
        f = kq[j]
        for s in rs:
            f *= Yq[s]
        for s in set(ps):
            Fp[s] += ps.count(s) * f
        for s in set(rs):
            nu = rs.count(s)
            Fm[s] += nu * f
            # d/dY_s of Y_s^nu times the rest, divided appropriately: F-_s / Y_s
            rest = kq[j]
            for o in rs:
                if o != s:
                    rest *= Yq[o]
            kk[s] += nu * rest * Yq[s] ** (nu - 1)
    return Fp, Fm, kk


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_rhs_exact_rationals(oracle_mod, seed):
    # small network with 1-, 2- and 3-body reactions, a repeated reactant and a
    # repeated product, one species at zero abundance
    A = [1, 1, 2, 3, 4]
    reactions = [((0,), (1,)), ((0, 1), (2,)), ((2,), (0, 1)), ((0, 0), (2,)),
                 ((0, 0, 1), (3,)), ((3,), (1, 1, 0)), ((2, 2), (4,)), ((4,), (2, 2)),
                 ((1, 2), (3,))]
    rng = np.random.default_rng(seed)
    net = custom_network(A, reactions, rng.uniform(-3, 3, len(reactions)), [0.0] * len(reactions))
    orc = oracle_mod.Oracle(net)
    k = np.exp(rng.uniform(-2, 4, len(reactions)))
    Y = rng.uniform(0.0, 0.5, 5)
    Y[3] = 0.0
    Fp, kk, f = orc.rhs(k, Y)
    eFp, eFm, ekk = _exact_rhs(net, k, Y)
    for i in range(5):
        assert abs(Fraction(float(Fp[i])) - eFp[i]) <= abs(eFp[i]) * Fraction(1, 2 ** 48) + Fraction(1, 2 ** 1000)
        assert abs(Fraction(float(kk[i])) - ekk[i]) <= abs(ekk[i]) * Fraction(1, 2 ** 48) + Fraction(1, 2 ** 1000)
        # F-_i = k_i Y_i (Eq. 1) holds for the oracle's k_i
        assert abs(Fraction(float(kk[i])) * Fraction(float(Y[i])) - eFm[i]) <= abs(eFm[i]) * Fraction(1, 2 ** 47) + Fraction(1, 2 ** 1000)
    # zero-abundance species still has a finite depletion rate from its 1st-order slots
    assert kk[3] > 0


def test_one_step_exact_rationals(oracle_mod):
    """A whole step (rhs + kappa switch) against Fractions, including one species
    on each branch."""
    net = custom_network([1, 1, 2], [((0,), (1,)), ((0, 1), (2,)), ((2,), (0, 1))],
                         [0.0, 0.0, 0.0], [0.0, 0.0, 0.0])
    orc = oracle_mod.Oracle(net)
    k = np.array([3.0, 40.0, 0.5])
    Y = np.array([0.25, 0.125, 0.25])
    dt = 0.25
    Fp, kk, _ = orc.rhs(k, Y)
    Yn, asy = orc.update(Y, Fp, kk, dt)
    eFp, _, ekk = _exact_rhs(net, k, Y)
    dq = Fraction(dt)
    for i in range(3):
        x = ekk[i] * dq
        if x >= 1:
            exp_ = (Fraction(Y[i]) + dq * eFp[i]) / (1 + x)
            assert asy[i]
        else:
            exp_ = Fraction(Y[i]) + dq * (eFp[i] - ekk[i] * Fraction(Y[i]))
            assert not asy[i]
        assert abs(Fraction(float(Yn[i])) - exp_) <= abs(exp_) * Fraction(1, 2 ** 49)
    assert asy.any() and (~asy).any()


# --------------------------------------------------------------------------
# Rate parameterisation and the T9, rho profile
# --------------------------------------------------------------------------
def test_rate_scaling_laws(oracle_mod):
    net = net150()
    orc = oracle_mod.Oracle(net)
    nr = net.n_reac
    k1 = orc.rates(1.0, 1.0)
    assert np.allclose(k1, np.exp(net.ln_k0), rtol=1e-15, atol=0)
    k2 = orc.rates(3.0, 1e8)
    kT = orc.rates(6.0, 1e8)
    assert np.allclose(kT / k2, 2.0 ** net.t9_exp, rtol=1e-13)
    kr = orc.rates(3.0, 1e9)
    assert np.allclose(kr / k2, 10.0 ** (nr - 1), rtol=1e-13)


def test_conditions_profile(oracle_mod):
    orc = oracle_mod.Oracle(pair_network(1.0, 1.0))
    T, r = orc.conditions(5.0, 1e8, 0.5, 0.5)
    assert T == pytest.approx(5.0 / math.e, rel=1e-15)
    assert r == pytest.approx(1e8 / math.e ** 3, rel=1e-15)
    assert orc.conditions(5.0, 1e8, 0.0, 123.0) == (5.0, 1e8)
    assert orc.conditions(5.0, 1e8, -1.0, 1.0) == (5.0, 1e8)


# --------------------------------------------------------------------------
# Conservation of sum_i A_i Y_i (Eq. 5.35: sum X = 1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("factory", [chain_network, net150, net365,
                                     lambda: random_tiny_network(6, 9, 4)])
def test_rhs_conserves_mass_number(oracle_mod, factory):
    net = factory()
    orc = oracle_mod.Oracle(net)
    rng = np.random.default_rng(0)
    for T9, rho in ((3.0, 1e8), (7.0, 1e9), (2.0, 1e7)):
        k = orc.rates(T9, rho)
        Y = rng.uniform(0, 1, net.n_species) * 10.0 ** rng.uniform(-12, 0, net.n_species)
        Fp, kk, _ = orc.rhs(k, Y)
        net_rate = np.sum(net.A * (Fp - kk * Y))
        scale = np.sum(net.A * (Fp + kk * Y))
        assert abs(net_rate) <= 1e-12 * scale


def test_forward_euler_only_run_conserves(oracle_mod):
    net = net150()
    orc = oracle_mod.Oracle(net)
    z = constant_zones(net)
    k = orc.rates(3.0, 1e8)
    _, kk, _ = orc.rhs(k, z.Y0[0])
    h = 0.2 / kk.max()
    # replay with kappa = inf: every species on the forward-Euler branch
    Y, _ = orc.replay(z, 0, np.full(200, h), opts=oracle_mod.OracleOpts(kappa=1e300))
    assert abs(np.sum(net.A * Y) - 1.0) <= 1e-12
    assert Y.min() >= 0.0


def test_full_run_drift_bounded_by_eps_c(oracle_mod):
    net = chain_network()
    orc = oracle_mod.Oracle(net)
    z = constant_zones(net)
    o = oracle_mod.OracleOpts()
    r = orc.integrate(z, 0, o, record=200000)
    assert r["status"] == 0 and r["t"] == z.t_end[0]
    drift = abs(np.sum(net.A * r["Y"]) - 1.0)
    assert drift <= r["steps"] * o.eps_c
    assert r["Y"].min() >= 0.0


# --------------------------------------------------------------------------
# Linear A <-> B: closed form, first-order convergence, exact linear maps
# --------------------------------------------------------------------------
def _pair_zone(t_end=1.0, t0=1e-6):
    from kn_inputs import Zones
    return Zones(Y0=np.array([[1.0, 0.0]]), T0=np.array([1.0]), rho0=np.array([1.0]),
                 tau=np.array([0.0]), t_start=np.array([t0]), t_end=np.array([t_end]),
                 dt_trial=np.array([t0]))


def test_pair_closed_form_and_order(oracle_mod):
    kf, kr = 3.0, 1.0
    net = pair_network(kf, kr)
    orc = oracle_mod.Oracle(net)
    z = _pair_zone(t_end=1.0)
    errs = []
    for er in (1e-2, 1e-3, 1e-4):
        r = orc.integrate(z, 0, oracle_mod.OracleOpts(eps_r=er, eps_c=1.0))
        assert r["status"] == 0
        yeq = kr / (kf + kr)
        ya = yeq + (1.0 - yeq) * math.exp(-(kf + kr) * (1.0 - 1e-6))
        errs.append(abs(r["Y"][0] - ya))
    # first order in eps_r: each 10x tighter tolerance gives about 10x smaller error
    for a, b in zip(errs, errs[1:]):
        assert 3.0 < a / b < 30.0
    assert errs[1] < 10 * 1e-3 * 1.0


def test_pair_fixed_dt_maps_are_matrix_powers(oracle_mod):
    kf, kr = 3.0, 1.0
    net = pair_network(kf, kr)
    orc = oracle_mod.Oracle(net)
    z = _pair_zone(t_end=1e9, t0=0.0)
    z.dt_trial[:] = 1.0
    Y0 = z.Y0[0]
    K = np.array([[-kf, kr], [kf, -kr]])
    # forward Euler on both (kf h, kr h < 1)
    h, n = 0.1, 37
    Y, _ = orc.replay(z, 0, np.full(n, h))
    ref = np.linalg.matrix_power(np.eye(2) + h * K, n) @ Y0
    assert np.allclose(Y, ref, rtol=1e-14, atol=0)
    # asymptotic on both (kf h, kr h >= 1): Y_A' = (Y_A + h kr Y_B)/(1 + kf h), ...
    h, n = 2.0, 25
    a, b = kf * h, kr * h
    M = np.array([[1 / (1 + a), h * kr / (1 + a)], [h * kf / (1 + b), 1 / (1 + b)]])
    Y, _ = orc.replay(z, 0, np.full(n, h))
    assert np.allclose(Y, np.linalg.matrix_power(M, n) @ Y0, rtol=1e-14, atol=0)
    # mixed: A asymptotic (kf h = 1.5), B forward Euler (kr h = 0.5)
    h, n = 0.5, 30
    M = np.array([[1 / (1 + kf * h), h * kr / (1 + kf * h)], [h * kf, 1 - kr * h]])
    Y, _ = orc.replay(z, 0, np.full(n, h))
    assert np.allclose(Y, np.linalg.matrix_power(M, n) @ Y0, rtol=1e-14, atol=1e-300)


# --------------------------------------------------------------------------
# Equilibrium of reversible pairs
# --------------------------------------------------------------------------
def test_pair_equilibrium_ratio(oracle_mod):
    """Fixed points of both branches satisfy k_f Y_A = k_r Y_B exactly: with a
    fixed dt the iteration contracts onto it (forward Euler factor |1-(kf+kr)h|,
    asymptotic factor |1 - kf kr h^2| / ((1 + kf h)(1 + kr h)))."""
    kf, kr = 5.0, 2.0
    net = pair_network(kf, kr)
    orc = oracle_mod.Oracle(net)
    z = _pair_zone(t_end=1e9, t0=0.0)
    for h, n in ((0.1, 80), (1.0, 80), (0.3, 80)):  # FE, asymptotic, mixed branches
        Y, _ = orc.replay(z, 0, np.full(n, h))
        assert Y[1] / Y[0] == pytest.approx(kf / kr, rel=1e-12)
    # the adaptive run heads to the same point
    z = _pair_zone(t_end=200.0)
    r = orc.integrate(z, 0, oracle_mod.OracleOpts(eps_r=1e-3, eps_c=1.0))
    assert r["status"] == 0
    assert r["Y"][1] / r["Y"][0] == pytest.approx(kf / kr, rel=1e-8)


def test_two_body_equilibrium(oracle_mod):
    """i + j <-> k with rho weighting on the 2-body direction: at the fixed
    point rho k0_f T9^n_f Y_i Y_j = k0_r T9^n_r Y_k (closed-form rates)."""
    from kn_inputs import Zones
    lf, lr = math.log(2e-8), math.log(3.0)
    net = custom_network([1, 1, 2], [((0, 1), (2,)), ((2,), (0, 1))], [lf, lr], [1.5, 0.5])
    orc = oracle_mod.Oracle(net)
    T9, rho = 2.0, 1e8
    z = Zones(Y0=np.array([[0.3, 0.5, 0.1]]), T0=np.array([T9]), rho0=np.array([rho]),
              tau=np.array([0.0]), t_start=np.array([0.0]), t_end=np.array([1e9]),
              dt_trial=np.array([0.05]))
    kfv = 2e-8 * T9 ** 1.5 * rho
    krv = 3.0 * T9 ** 0.5
    Y, _ = orc.replay(z, 0, np.full(400, 0.02))  # forward Euler, contracts onto the fixed point
    assert kfv * Y[0] * Y[1] == pytest.approx(krv * Y[2], rel=1e-10)
    assert np.sum(net.A * Y) == pytest.approx(1.0, abs=1e-14)
    # that point is also a fixed point of the asymptotic formula (Eq. 3): one
    # large step with every species asymptotic leaves it unchanged
    k = orc.rates(T9, rho)
    Fp, kk, _ = orc.rhs(k, Y)
    Yn, asy = orc.update(Y, Fp, kk, 50.0)
    assert asy.all()
    assert np.allclose(Yn, Y, rtol=1e-13, atol=0)


# --------------------------------------------------------------------------
# Dense LU against the library solver; backward Euler against closed forms
# --------------------------------------------------------------------------
def test_lu_matches_library_solver(oracle_mod):
    rng = np.random.default_rng(3)
    for n in (1, 3, 8, 40):
        J = rng.normal(size=(n, n)) + n * np.eye(n)
        b = rng.normal(size=n)
        x = oracle_mod.lu_solve(J, b)
        assert np.allclose(x, np.linalg.solve(J, b), rtol=1e-12, atol=1e-14)
    # a matrix that needs pivoting
    J = np.array([[0.0, 1.0], [1.0, 0.0]])
    assert np.allclose(oracle_mod.lu_solve(J, [2.0, 3.0]), [3.0, 2.0])


def test_backward_euler_linear_map(oracle_mod):
    kf, kr = 30.0, 10.0
    net = pair_network(kf, kr)
    orc = oracle_mod.Oracle(net)
    z = _pair_zone(t_end=1.0, t0=0.0)
    n = 20
    Y, it = orc.be_fixed(z, 0, n)
    assert it >= 1
    K = np.array([[-kf, kr], [kf, -kr]])
    h = 1.0 / n
    ref = np.linalg.matrix_power(np.linalg.inv(np.eye(2) - h * K), n) @ z.Y0[0]
    assert np.allclose(Y, ref, rtol=1e-12)


def test_backward_euler_newton_solves_nonlinear_step(oracle_mod):
    net = random_tiny_network(6, 9, 11)
    orc = oracle_mod.Oracle(net)
    k = orc.rates(1.0, 1.0) * 50.0
    Y0 = net.initial_Y()
    h = 0.3
    Y, it = orc.be_step(k, Y0, h)
    assert it > 0
    Fp, kk, _ = orc.rhs(k, Y)
    resid = Y - Y0 - h * (Fp - kk * Y)
    assert np.max(np.abs(resid)) < 1e-13


@pytest.mark.parametrize("n_sp,n_rx,seed", [(3, 3, 1), (4, 6, 2), (5, 8, 3), (6, 10, 5), (8, 14, 6)])
def test_explicit_vs_backward_euler_richardson(oracle_mod, n_sp, n_rx, seed):
    """Brute force on tiny networks: dense-LU backward Euler with fixed small
    steps, Richardson-extrapolated (first order: 2 Y(h/2) - Y(h)), is the truth.
    The explicit oracle converges to it as eps_r tightens: within 3e-2 at
    eps_r = 1e-3 and 1e-3 at eps_r = 1e-4, relative, on abundances above 1e-10."""
    from kn_inputs import Zones
    net = random_tiny_network(n_sp, n_rx, seed)
    orc = oracle_mod.Oracle(net)
    z = Zones(Y0=net.initial_Y()[None, :], T0=np.array([1.0]), rho0=np.array([1.0]),
              tau=np.array([0.0]), t_start=np.array([0.0]), t_end=np.array([0.5]),
              dt_trial=np.array([1e-6]))
    n = 40000
    Y1, it1 = orc.be_fixed(z, 0, n)
    Y2, it2 = orc.be_fixed(z, 0, 2 * n)
    assert it1 > 0 and it2 > 0
    truth = 2.0 * Y2 - Y1
    m = truth > 1e-10
    assert m.sum() >= 2
    # the Richardson correction is a small fraction of the abundance
    assert np.max(np.abs(Y2[m] - truth[m]) / truth[m]) < 1e-2
    errs = []
    for er, bound in ((1e-3, 3e-2), (1e-4, 1e-3)):
        r = orc.integrate(z, 0, oracle_mod.OracleOpts(eps_r=er, eps_c=1e-5))
        assert r["status"] == 0
        errs.append(np.max(np.abs(r["Y"][m] - truth[m]) / truth[m]))
        assert errs[-1] < bound
    assert errs[1] <= max(errs[0], 1e-4)  # tighter tolerance: no worse (both may be tiny)


# --------------------------------------------------------------------------
# The step loop: replay reproduces a recorded run; every accepted step passed
# --------------------------------------------------------------------------
def test_replay_reproduces_and_every_step_passes(oracle_mod):
    net = net150()
    orc = oracle_mod.Oracle(net)
    z = profile_zones(net, 2, t_end=3e-11)
    o = oracle_mod.OracleOpts()
    r = orc.integrate(z, 1, o, record=10 ** 6)
    assert r["status"] == 0 and r["t"] == z.t_end[1]
    dts = r["dts"]
    assert len(dts) == r["steps"]
    Yr, tr = orc.replay(z, 1, dts)
    assert np.array_equal(Yr, r["Y"]) and tr == r["t"]
    # step-by-step: every accepted step satisfies the accept test
    Y = z.Y0[1].copy()
    t = z.t_start[1]
    for h in dts[:300]:
        T9, rho = orc.conditions(z.T0[1], z.rho0[1], z.tau[1], t)
        Yn, _ = orc.step(Y, T9, rho, h)
        acc, cons, rel, fin = orc.test(Y, Yn, o)
        assert acc and cons <= o.eps_c and rel <= o.eps_r
        Y, t = Yn, t + h


def test_positivity_and_status_on_batch(oracle_mod):
    net = net150()
    orc = oracle_mod.Oracle(net)
    z = profile_zones(net, 4, t_end=1e-11)
    r = orc.integrate_batch(z, threads=2)
    assert (r["status"] == 0).all()
    assert (r["Y"] >= 0).all()
    assert np.all(r["t"] == z.t_end)


def test_status_codes(oracle_mod):
    net = net150()
    orc = oracle_mod.Oracle(net)
    z = constant_zones(net, t_end=1e-9)
    r = orc.integrate(z, 0, oracle_mod.OracleOpts(max_steps=50))
    assert r["status"] == 1 and r["steps"] == 50
    r = orc.integrate(z, 0, oracle_mod.OracleOpts(max_reject=0, grow_max=1e6, safety=1e6))
    assert r["status"] == 4
    zz = constant_zones(net, t_end=1e-9)
    zz.Y0[0, 5] = np.nan
    r = orc.integrate(zz, 0, oracle_mod.OracleOpts(max_reject=3))
    assert r["status"] == 3


def test_energy_release_telescopes(oracle_mod):
    """sum_i B_i (Y_end - Y_start) equals sum over steps of dt sum_j Q_j f_j,
    Q_j = sum_products B - sum_reactants B, exactly under forward Euler (every
    species on that branch), since dY_i = dt sum_j nu_ij f_j."""
    from kn_inputs import binding_energies
    net = net150()
    orc = oracle_mod.Oracle(net)
    B = binding_energies(net)
    Q = np.array([B[p[p >= 0]].sum() - B[r[r >= 0]].sum() for r, p in zip(net.reac, net.prod)])
    z = constant_zones(net)
    k = orc.rates(3.0, 1e8)
    _, kk, _ = orc.rhs(k, z.Y0[0])
    h = 0.2 / kk.max()
    Y = z.Y0[0].copy()
    flux_sum = 0.0
    for _ in range(50):
        _, _, f = orc.rhs(k, Y)
        flux_sum += h * float(np.dot(Q, f))
        Y, _ = orc.replay(type(z)(Y0=Y[None, :], T0=z.T0, rho0=z.rho0, tau=z.tau, t_start=z.t_start,
                                   t_end=np.array([1.0]), dt_trial=z.dt_trial), 0, [h],
                          opts=oracle_mod.OracleOpts(kappa=1e300))
    assert float(np.dot(B, Y - z.Y0[0])) == pytest.approx(flux_sum, rel=1e-9)
