"""Pins of the oracle's alpha-QSS update (the explicit QSS alternative to
Eq. 3 that Sec. 11 proposes; the formula is the alpha-QSS predictor-corrector
of Mott, Oran & van Leer, J. Comput. Phys. 164 (2000) 407).

Each check compares the oracle with mathematics it does not contain:
- alpha against the exact function 1/(1 - e^-x) - 1/x (high-precision, from
  mpmath) near 0, at 1 and for large x;
- one step of a linear decay against e^-x, which the scheme matches to
  O(x^7) because alpha matches the exact function to O(x^5);
- a species with no depletion takes the trapezoidal rule;
- the update as evaluated (without the printed form's cancellation) against
  the printed form in 50-digit arithmetic;
- second-order convergence on a nonlinear network (2a -> b, closed form) and
  on a decay with time-dependent rates (closed form), which fails if the
  corrector is dropped or the predicted state's rates are taken at t;
- the whole controller with method QSS: the A <-> B pair reaches its
  equilibrium ratio and the accepted steps pass the accept test.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from kn_inputs import Zones, custom_network, pair_network

mpmath = pytest.importorskip("mpmath")


def _alpha_exact(x):
    mpmath.mp.dps = 50
    X = mpmath.mpf(x)
    return float(1 / (1 - mpmath.e ** (-X)) - 1 / X)


def test_alpha_limits_and_series(oracle_mod):
    a = oracle_mod.Oracle.qss_alpha
    assert a(0.0) == 0.5  # the trapezoidal limit
    assert a(1e300) == 1.0  # the stiff limit
    # the exact alpha is 1/2 + x/12 - x^3/720 + x^5/30240 - ...; the rational
    # approximation agrees through x^4 (its x^5 coefficient is 1/21600)
    for x in (1e-3, 1e-2, 0.1, 0.25, 0.5):
        err = abs(a(x) - _alpha_exact(x))
        assert err <= 2e-5 * x ** 5 + 1e-16, (x, err)
    # a slip in any coefficient of the rational function breaks the x^2 term
    x = 0.1
    assert abs(a(x) - (0.5 + x / 12 - x ** 3 / 720)) < 1e-9
    # large x: both are 1 - 1/x + O(1/x^2) (the approximation's 1/x^2
    # coefficient is 12, the exact one's 0)
    for x in (100.0, 1e3, 1e4):
        assert abs(a(x) - _alpha_exact(x)) <= 13.0 / x ** 2, x


def test_alpha_monotone_between_limits(oracle_mod):
    a = oracle_mod.Oracle.qss_alpha
    xs = np.logspace(-6, 8, 400)
    v = np.array([a(x) for x in xs])
    assert np.all(v > 0.5) and np.all(v < 1.0)
    assert np.all(np.diff(v) >= 0.0)
    # continuous where the evaluation switches between powers of x and of 1/x
    assert abs(a(1.0) - a(np.nextafter(1.0, 2.0))) < 1e-15


def _literal_update(Y, F, k, dt):
    """The scheme's update Y + dt (F - k Y) / (1 + alpha x), x = k dt, with
    alpha's rational function, as printed, in 50-digit arithmetic."""
    mpmath.mp.dps = 50
    Y, F, k, dt = (mpmath.mpf(float(v)) for v in (Y, F, k, dt))
    x = k * dt
    if x == 0:
        a = mpmath.mpf(1) / 2
    else:
        r = 1 / x
        a = (180 * r ** 3 + 60 * r ** 2 + 11 * r + 1) / (360 * r ** 3 + 60 * r ** 2 + 12 * r + 1)
    return Y + dt * (F - k * Y) / (1 + a * x)


def test_update_matches_the_formula_in_50_digits(oracle_mod):
    """The oracle evaluates the update without the cancellation of the printed
    form (the two agree algebraically); against the printed form in 50-digit
    arithmetic it is within a few ulp for k dt from 1e-8 to 1e12, where the
    printed form in FP64 loses up to all of its digits."""
    O = oracle_mod.Oracle(_decay_net())
    rng = np.random.default_rng(17)
    worst = 0.0
    for _ in range(400):
        x = 10.0 ** rng.uniform(-8, 12)
        dt = 10.0 ** rng.uniform(-12, -3)
        k = x / dt
        Y = np.array([10.0 ** rng.uniform(-12, 0), 0.0])
        F = np.array([10.0 ** rng.uniform(-6, 6) * (k * Y[0] if rng.uniform() < 0.5 else 1.0), 0.0])
        kk = np.array([k, 0.0])
        got = O.qss_predict(Y, F, kk, dt)[0]
        want = float(_literal_update(Y[0], F[0], k, dt))
        worst = max(worst, abs(got - want) / abs(want))
        # the corrector with kbar = k and F+p = F+0 = F takes the same update
        got_c = O.qss_correct(Y, F, kk, F, kk, dt)[0]
        assert abs(got_c - want) <= 1e-14 * abs(want)
    assert worst <= 1e-14, worst


def _decay_net():
    # a -> b, k = 1 (ln k0 = 0, n = 0), A = (1, 1)
    return custom_network([1.0, 1.0], [((0,), (1,))], [0.0], [0.0])


@pytest.mark.parametrize("x", [0.05, 0.1, 0.2, 0.5])
def test_linear_decay_step_matches_exponential(oracle_mod, x):
    """One step of a -> b from Y = (1, 0) with k dt = x: the exact step of
    dY/dt = -k Y is e^-x, and the scheme's differs from it by
    x^2 (alpha - alpha_exact) / ((1 + alpha x)(1 + alpha_exact x)) = O(x^7)."""
    O = oracle_mod.Oracle(_decay_net())
    Yc, Fp0, k0, Yp = O.qss_step(np.array([1.0, 0.0]), 1.0, 1.0, x)
    assert k0[0] == 1.0 and Fp0[0] == 0.0
    assert abs(Yc[0] - math.exp(-x)) <= 3e-5 * x ** 7 + 4e-16
    # k of species a does not depend on Y, so the corrector repeats the predictor
    assert Yc[0] == Yp[0]
    # species b has no depletion: alpha(0) = 1/2, the trapezoidal rule
    assert Yc[1] == pytest.approx(x * (1.0 + Yp[0]) / 2.0, rel=4e-16, abs=0)


@pytest.mark.parametrize("x", [1.0, 10.0, 1e3, 1e8])
def test_linear_decay_stiff_step_bounded(oracle_mod, x):
    """Far past the stability limit of an explicit Euler step (k dt >> 1) the
    QSS step stays in [0, 1] and decays toward the equilibrium 0."""
    O = oracle_mod.Oracle(_decay_net())
    Yc, _, _, _ = O.qss_step(np.array([1.0, 0.0]), 1.0, 1.0, x)
    assert 0.0 <= Yc[0] <= 1.0
    assert Yc[0] <= 1.0 / (1.0 + 0.5 * x)


def _replay_error(oracle_mod, net, Y0, exact, tau, T, n):
    z = Zones(Y0=np.array([Y0]), T0=np.array([1.0]), rho0=np.array([1.0]), tau=np.array([tau]),
              t_start=np.array([0.0]), t_end=np.array([T]), dt_trial=np.array([T / n]))
    Y, t = oracle_mod.Oracle(net).replay(z, 0, np.full(n, T / n), oracle_mod.OracleOpts(method=1))
    assert t == T
    return abs(Y[0] - exact)


def test_second_order_nonlinear(oracle_mod):
    """2a -> b with k = 1: dY_a/dt = -2 Y_a^2, Y_a(t) = Y0 / (1 + 2 Y0 t).
    Halving dt divides the error by 4 (second order); Eq. (3) divides it by 2."""
    net = custom_network([1.0, 2.0], [((0, 0), (1,))], [0.0], [0.0])
    exact = 1.0 / (1.0 + 2.0)
    errs = [_replay_error(oracle_mod, net, [1.0, 0.0], exact, 0.0, 1.0, n) for n in (16, 32, 64, 128)]
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.8 < r < 4.2 for r in ratios), ratios


def test_second_order_time_dependent_rates(oracle_mod):
    """a -> b with k(t) = T9(t)^2, T9 = e^{-t/tau}, tau = 1:
    Y_a(T) = exp(-(1 - e^{-2T}) / 2).  Second order needs the predicted
    state's rates at t + dt (at t the order drops to one)."""
    net = custom_network([1.0, 1.0], [((0,), (1,))], [0.0], [2.0])
    exact = math.exp(-(1.0 - math.exp(-2.0)) / 2.0)
    errs = [_replay_error(oracle_mod, net, [1.0, 0.0], exact, 1.0, 1.0, n) for n in (8, 16, 32, 64)]
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.8 < r < 4.2 for r in ratios), ratios


def test_controller_qss_reaches_equilibrium(oracle_mod):
    """A <-> B with k_f = 2, k_r = 1 under the step controller with method
    QSS: Y_b / Y_a -> k_f / k_r, every recorded step passes the accept test
    on replay, and the run ends ok."""
    net = pair_network(2.0, 1.0)
    O = oracle_mod.Oracle(net)
    z = Zones(Y0=np.array([[1.0, 0.0]]), T0=np.array([1.0]), rho0=np.array([1.0]), tau=np.array([0.0]),
              t_start=np.array([1e-3]), t_end=np.array([30.0]), dt_trial=np.array([1e-3]))
    opts = oracle_mod.OracleOpts(method=1, eps_r=0.05, eps_c=1e-3)
    r = O.integrate(z, 0, opts, record=100000)
    assert r["status"] == 0 and r["t"] == 30.0
    # the exact equilibrium is a fixed point of the QSS map for every dt, but
    # at k dt >> 1 the pair's deviation mode is barely damped (the predictor
    # tends to the QSS limit, which swaps the deviation's sign), so the ratio
    # keeps what the controller's last small steps left: 1.2e-5 here, as
    # Eq. (3) leaves 2e-6
    assert r["Y"][1] / r["Y"][0] == pytest.approx(2.0, rel=1e-4)
    # mass is not conserved exactly by either update; the controller bounds
    # each step's drift by eps_c
    assert abs(r["Y"].sum() - 1.0) <= r["steps"] * 1e-3
    # replaying the recorded steps one by one, each passes the accept test
    Y = np.array([1.0, 0.0])
    t = 1e-3
    for h in r["dts"][:200]:
        Yn, _, _, _ = O.qss_step(Y, 1.0, 1.0, h)
        ok, cons, rel, fin = O.test(Y, Yn, opts)
        assert ok
        Y, t = Yn, t + h
