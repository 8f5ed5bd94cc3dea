"""GPU parity of the alpha-QSS update (KN_METHOD_QSS, FP64 and mixed forms)
against the oracle's FP64 QSS (the alternative to Eq. 3 that Sec. 11
proposes).

Tiers as for Eq. 3:
  1. one step from identical states (kn_probe_step): F+ and k of the start
     state, and Y' element by element;
  2. the oracle's accepted dt sequence replayed: end states element by
     element at 1e-9 (the FP64 bar);
  3. free-running: the GPU's controller against the oracle's, step counts
     within 2 % and end states within 10 eps_r.

Tolerances as for Eq. 3: FP64 1e-12 one step, 1e-9 replayed; mixed 1e-5 and
1e-4 (FP32 rates, fluxes, gathers and predictor; float-float pairs).  Both sides
evaluate the update y + h (f - k y)/(1 + alpha k h) in the form without
cancellation (c0 y + c1 h f)/c2; printed as a difference, the predictor of a
species destroyed with k h >> 1 would keep a relative error of about
eps (k h)^2 / 12, and rounding differences would reach Y' amplified (up to
1e-6 on these inputs, against 4e-15 with the form used).
"""
import numpy as np
import pytest

from kn_inputs import (Zones, chain_network, constant_zones, net150, net365, profile_zones)

pytestmark = pytest.mark.gpu

FP64, MIXED, M64 = 0, 1, 2
QSS = 1
TOL_STEP = {FP64: 1e-12, MIXED: 1e-5}
TOL_REPLAY = {FP64: 1e-9, MIXED: 1e-4}


@pytest.fixture(scope="module")
def kn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_5826_gb300 import build, kn as knmod
    build.build()
    return knmod


def _rel_err(a, b, floor):
    m = np.abs(b) > floor
    if not m.any():
        return 0.0
    return float(np.max(np.abs(a[m] - b[m]) / np.abs(b[m])))


def _random_states(net, Z, seed):
    rng = np.random.default_rng(seed)
    Y = 10.0 ** rng.uniform(-14, 0, (Z, net.n_species))
    Y[rng.uniform(size=Y.shape) < 0.1] = 0.0
    Y /= (Y * net.A).sum(1, keepdims=True)
    return Y


def _oracle_qss_step(orc, Y, k, kq, dt):
    Fp0, k0, _ = orc.rhs(k, Y)
    Yp = orc.qss_predict(Y, Fp0, k0, dt)
    Fpp, kp, _ = orc.rhs(kq, Yp)
    return orc.qss_correct(Y, Fp0, k0, Fpp, kp, dt), Fp0, k0


@pytest.mark.parametrize("prec", [FP64, MIXED])
@pytest.mark.parametrize("factory", [chain_network, net150, net365])
@pytest.mark.parametrize("tiling", [(0, 0), (32, 32), (128, 256)])
def test_qss_one_step_parity(kn, oracle_mod, prec, factory, tiling):
    net = factory()
    orc = oracle_mod.Oracle(net)
    Z = 37
    Y = _random_states(net, Z, 5)
    rng = np.random.default_rng(1)
    T0 = rng.uniform(2, 7, Z)
    rho0 = 10 ** rng.uniform(7, 9, Z)
    tau = np.where(np.arange(Z) % 3 == 0, 0.0, 10 ** rng.uniform(-1, 0, Z))
    ts = 10 ** rng.uniform(-12, -9, Z)
    dt = 10 ** rng.uniform(-16, -9, Z)
    z = Zones(Y0=Y, T0=T0, rho0=rho0, tau=tau, t_start=ts, t_end=np.ones(Z), dt_trial=dt)
    g = kn.Network(net)
    g.set_zones(z)
    G, P = tiling
    if prec == FP64 and net.n_species == 365 and P > G:
        with pytest.raises(kn.KnError, match="no tiling fits"):
            g.probe(kn.Opts(precision=prec, method=QSS, threads_per_zone=G, threads_per_cta=P))
        return
    out = g.probe(kn.Opts(precision=prec, method=QSS, threads_per_zone=G, threads_per_cta=P))
    tol = TOL_STEP[prec]
    for i in range(Z):
        T9, rho = orc.conditions(T0[i], rho0[i], tau[i], ts[i])
        T9p, rhop = orc.conditions(T0[i], rho0[i], tau[i], ts[i] + dt[i])
        k, kq = orc.rates(T9, rho), orc.rates(T9p, rhop)
        Yc, Fp0, k0 = _oracle_qss_step(orc, Y[i], k, kq, dt[i])
        floor = 1e-300 if prec == FP64 else 1e-30 * max(Fp0.max(), 1e-300)
        assert _rel_err(out["Fp"][i], Fp0, floor) < tol, ("F+", i)
        floor = 1e-300 if prec == FP64 else 1e-30 * max(k0.max(), 1e-300)
        assert _rel_err(out["k"][i], k0, floor) < tol, ("k", i)
        scale = np.maximum(Y[i], Yc)
        m = scale > (1e-30 if prec == FP64 else 1e-10)
        err = float(np.max(np.abs(out["Y1"][i][m] - Yc[m]) / scale[m]))
        assert err < tol, ("Y1", i, err)
        acc, cons, rel, fin = orc.test(Y[i], Yc)
        gross = np.sum(np.abs(net.A * (Yc - Y[i])))
        assert abs(out["cons"][i] - cons) <= 10 * tol * gross + 1e-15, ("cons", i)
        assert abs(out["rel"][i] - rel) <= (1e-10 if prec == FP64 else 10 * tol), ("rel", i)


def _replay(kn, net, zones, dts_list, prec):
    import torch
    g = kn.Network(net)
    g.set_zones(zones)
    lens = np.array([len(d) for d in dts_list], np.int64)
    off = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    flat = np.concatenate(dts_list) if lens.sum() else np.zeros(1)
    dev = torch.device("cuda")
    t_dt = torch.from_numpy(flat).to(dev)
    t_off = torch.from_numpy(off).to(dev)
    t_len = torch.from_numpy(lens).to(dev)
    o = kn.Opts(precision=prec, method=QSS, replay_dt=t_dt.data_ptr(), replay_off=t_off.data_ptr(),
                replay_len=t_len.data_ptr())
    kn.integrate_batch([g], o)
    r = g.get()
    del t_dt, t_off, t_len
    return r


@pytest.mark.parametrize("prec", [FP64, MIXED])
@pytest.mark.parametrize("case", ["chain_constant", "chain_profiles", "net150_profiles"])
def test_qss_replay_parity(kn, oracle_mod, prec, case):
    if case == "chain_constant":
        net = chain_network()
        z = constant_zones(net)
    elif case == "chain_profiles":
        net = chain_network()
        z = profile_zones(net, 6, t_end=1e-3)
    else:
        net = net150()
        z = profile_zones(net, 6, t_end=1e-10)
    orc = oracle_mod.Oracle(net)
    opts = oracle_mod.OracleOpts(method=QSS)
    rec = [orc.integrate(z, i, opts, record=10 ** 6) for i in range(z.n_zones)]
    r = _replay(kn, net, z, [x["dts"] for x in rec], prec)
    for i in range(z.n_zones):
        assert r["status"][i] == 0 and r["steps"][i] == rec[i]["steps"]
        assert r["t"][i] == rec[i]["t"]
        err = _rel_err(r["Y"][i], rec[i]["Y"], 1e-10)
        assert err < TOL_REPLAY[prec], (i, err)


@pytest.mark.parametrize("prec", [FP64, MIXED])
@pytest.mark.parametrize("case", ["chain_profiles", "net150_profiles"])
def test_qss_free_running(kn, oracle_mod, prec, case):
    if case == "chain_profiles":
        net = chain_network()
        z = profile_zones(net, 12, t_end=1e-2)
    else:
        net = net150()
        z = profile_zones(net, 8, t_end=1e-10)
    orc = oracle_mod.Oracle(net)
    opts = oracle_mod.OracleOpts(method=QSS)
    g = kn.Network(net)
    g.set_zones(z)
    kn.integrate_batch([g], kn.Opts(precision=prec, method=QSS))
    r = g.get()
    for i in range(z.n_zones):
        o = orc.integrate(z, i, opts)
        assert r["status"][i] == 0 and o["status"] == 0
        assert r["t"][i] == o["t"]
        assert abs(r["steps"][i] - o["steps"]) <= 0.02 * o["steps"] + 2, (i, r["steps"][i], o["steps"])
        assert _rel_err(r["Y"][i], o["Y"], 1e-10) < 10 * 0.05, i


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_qss_differs_from_asymptotic_and_is_deterministic(kn, prec):
    """The method switch reaches the kernel: QSS and Eq. 3 take different step
    counts on the chain, and two QSS runs agree bit for bit."""
    net = chain_network()
    z = profile_zones(net, 8, t_end=1e-3)
    res = []
    for method in (0, QSS, QSS):
        g = kn.Network(net)
        g.set_zones(z)
        kn.integrate_batch([g], kn.Opts(precision=prec, method=method))
        res.append(g.get())
    assert not np.array_equal(res[0]["steps"], res[1]["steps"])
    assert np.array_equal(res[1]["steps"], res[2]["steps"])
    assert np.array_equal(res[1]["Y"], res[2]["Y"])


def test_qss_refuses_other_forms(kn):
    net = chain_network()
    g = kn.Network(net)
    g.set_zones(constant_zones(net))
    with pytest.raises(kn.KnError, match="KN_METHOD_QSS"):
        kn.integrate_batch([g], kn.Opts(precision=M64, method=QSS))
    with pytest.raises(kn.KnError, match="opts.method"):
        kn.integrate_batch([g], kn.Opts(precision=FP64, method=7))


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_qss_operator_split_and_energy(kn, oracle_mod, prec):
    """The hydro-split driver (Sec. 4 and 6: conditions held per interval, the
    last dt carried over) with the QSS update: every interval against the
    oracle's QSS from the oracle's own previous state, and the energy
    release of each interval."""
    from kn_inputs import binding_energies
    from paper_1409_5826_gb300 import opsplit
    net = net150()
    B = binding_energies(net)
    Z = 8
    z = profile_zones(net, Z, t_end=1e-11)
    edges = [1e-12, 4e-12, 1e-11, 2e-11]
    schedule = [(z.T0 * (1 - 0.04 * k), z.rho0 * (1 - 0.08 * k), np.full(Z, edges[k + 1]))
                for k in range(len(edges) - 1)]
    g = kn.Network(net)
    g.set_binding_energies(B)
    res = opsplit.run(g, z, schedule, kn.Opts(precision=prec, method=QSS))
    orc = oracle_mod.Oracle(net)
    opts = oracle_mod.OracleOpts(method=QSS)
    for i in range(Z):
        Y = z.Y0[i].copy()
        dt = z.dt_trial[i]
        for k, (T9, rho, te) in enumerate(schedule):
            zk = Zones(Y0=Y[None, :], T0=np.array([T9[i]]), rho0=np.array([rho[i]]), tau=np.zeros(1),
                       t_start=np.array([edges[k]]), t_end=np.array([te[i]]), dt_trial=np.array([dt]))
            r = orc.integrate(zk, 0, opts)
            assert r["status"] == 0
            got = res[k]
            assert got["status"][i] == 0 and got["t"][i] == te[i]
            assert _rel_err(got["Y"][i], r["Y"], 1e-10) < 10 * 0.05
            y_before = z.Y0[i] if k == 0 else res[k - 1]["Y"][i]
            assert got["energy"][i] == pytest.approx(float(B @ (got["Y"][i] - y_before)), rel=1e-9, abs=1e-12)
            e_ref = float(B @ (r["Y"] - Y))
            assert got["energy"][i] == pytest.approx(e_ref, rel=0.05, abs=1e-3 * abs(e_ref) + 1e-6)
            Y, dt = r["Y"], r["dt_next"]


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_qss_edge_cases(kn, oracle_mod, prec):
    """Statuses through the QSS path: invalid device inputs, the step limit
    (with the end state of the oracle's QSS after the same 50 steps), the
    reject limit, dt underflow, and an interval shorter than the trial dt."""
    import torch
    net = net150()
    g = kn.Network(net)
    z = constant_zones(net, 3, t_end=1e-11)
    dz = {k: torch.from_numpy(np.ascontiguousarray(getattr(z, k))).cuda()
          for k in ("Y0", "T0", "rho0", "tau", "t_start", "t_end", "dt_trial")}
    dz["Y0"][1, 7] = float("nan")
    dz["rho0"][2] = -1.0
    g.set_zones(dz)
    kn.integrate_batch([g], kn.Opts(precision=prec, method=QSS))
    assert g.get()["status"].tolist() == [0, 5, 5]
    z = constant_zones(net, 3, t_end=1e-9)
    g.set_zones(z)
    kn.integrate_batch([g], kn.Opts(precision=prec, method=QSS, max_steps=50))
    r = g.get()
    assert (r["status"] == 1).all() and (r["steps"] == 50).all()
    assert (r["t"] < z.t_end).all()
    ref = oracle_mod.Oracle(net).integrate(z, 0, oracle_mod.OracleOpts(method=QSS, max_steps=50))
    assert ref["status"] == 1 and ref["steps"] == 50
    assert _rel_err(r["Y"][0], ref["Y"], 1e-10) < (1e-9 if prec == FP64 else 10 * 0.05)
    g.set_zones(z)
    kn.integrate_batch([g], kn.Opts(precision=prec, method=QSS, max_reject=0, grow_max=1e6, safety=1e6))
    r = g.get()
    assert (r["status"] == 4).all() and (r["rejects"] >= 1).all()
    # a reject whose halved step falls below dt_min_frac * t: DT_UNDERFLOW
    g.set_zones(z)
    kn.integrate_batch([g], kn.Opts(precision=prec, method=QSS, dt_min_frac=0.9))
    r = g.get()
    ref = oracle_mod.Oracle(net).integrate(z, 0, oracle_mod.OracleOpts(method=QSS, dt_min_frac=0.9))
    assert ref["status"] == 2 and (r["status"] == 2).all()
    z = constant_zones(net, 1, t_end=1e-12 + 1e-15)
    g.set_zones(z)
    kn.integrate_batch([g], kn.Opts(precision=prec, method=QSS))
    r = g.get()
    ref = oracle_mod.Oracle(net).integrate(z, 0, oracle_mod.OracleOpts(method=QSS))
    assert r["status"][0] == 0 and r["t"][0] == z.t_end[0] == ref["t"]
    assert abs(r["steps"][0] - ref["steps"]) <= max(2, (0.02 if prec == FP64 else 0.05) * ref["steps"])
