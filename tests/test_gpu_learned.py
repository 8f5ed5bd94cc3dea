"""GPU checks of the learned timestep proposal.

1. Records: the integrator, replaying the oracle's dt sequence in FP64, writes
   features and labels at every accepted state; the oracle computes the same
   from its own states (oracle/mlp.py).  Histogram counts are integers, so
   the quantile features agree exactly unless a value sits on a binary-
   exponent boundary; labels agree unless a grid step sits on the accept
   threshold.  Both mismatch rates must stay below 2 %.
2. Learned mode: a network trained on the integrator's own records proposes
   dt; the plain controller judges every step, so the end states stay within
   the free-running tolerance of the oracle and every zone finishes.
3. Gain: trained on records from training zones, evaluated on fresh-seed
   zones against the plain controller at equal accuracy (end-state error
   against a tight-tolerance oracle run); the measured gain is printed.
"""
import math
import time

import numpy as np
import pytest

import oracle.mlp as M
from kn_inputs import chain_network, constant_zones, net150, profile_zones

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_5826_gb300 import build, kn, learned
    build.build()
    return torch, kn, learned


def _oracle_records(orc, z, dts):
    Y = z.Y0[0].copy()
    t = z.t_start[0]
    feats, labels = [], []
    for i, h in enumerate(dts):
        T9, rho = orc.conditions(z.T0[0], z.rho0[0], z.tau[0], t)
        Y, _ = orc.step(Y, T9, rho, h)
        t = z.t_end[0] if h >= z.t_end[0] - t else t + h
        if i == len(dts) - 1:
            break
        T9, rho = orc.conditions(z.T0[0], z.rho0[0], z.tau[0], t)
        Fp, kk, _ = orc.rhs(orc.rates(T9, rho), Y)
        feats.append(M.features(math.log(T9), math.log(rho), h, Y, Fp, kk))
        labels.append(M.label(orc, Y, Fp, kk, h, t, z.t_end[0]))
    return np.array(feats), np.array(labels, np.float32)


@pytest.mark.parametrize("which", ["chain", "net150", "net150_profile"])
def test_records_match_oracle(env, oracle_mod, which):
    torch, kn, learned = env
    if which == "chain":
        net = chain_network()
        z = constant_zones(net, t_end=3e-9)
    elif which == "net150":
        net = net150()
        z = constant_zones(net, t_end=2e-11)
    else:
        net = net150()
        z = profile_zones(net, 1, base_seed=4242, t_end=2e-11)
    orc = oracle_mod.Oracle(net)
    rec = orc.integrate(z, 0, record=10 ** 6)
    dts = rec["dts"]
    ref_f, ref_l = _oracle_records(orc, z, dts)
    g = kn.Network(net)
    g.set_zones(z)
    dev = torch.device("cuda")
    cap = len(dts) + 8
    feat = torch.full((cap, 64), float("nan"), dtype=torch.float32, device=dev)
    lab = torch.full((cap,), float("nan"), dtype=torch.float32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    t_dt = torch.from_numpy(dts).to(dev)
    t_off = torch.zeros(1, dtype=torch.int64, device=dev)
    t_len = torch.tensor([len(dts)], dtype=torch.int64, device=dev)
    o = kn.Opts(precision=kn.PREC_FP64, replay_dt=t_dt.data_ptr(), replay_off=t_off.data_ptr(),
                replay_len=t_len.data_ptr(), record_features=feat.data_ptr(), record_labels=lab.data_ptr(),
                record_capacity=cap, record_count=cnt.data_ptr())
    kn.integrate_batch([g], o)
    torch.cuda.synchronize()
    n = int(cnt.item())
    assert n == len(dts) - 1 == len(ref_l)
    gf = feat[:n].cpu().numpy()
    gl = lab[:n].cpu().numpy()
    # scalars: ln T9, ln rho, ln dt_prev, asymptotic fraction
    assert np.allclose(gf[:, :3], ref_f[:, :3], rtol=1e-5, atol=1e-5)
    assert np.mean(np.abs(gf[:, 3] - ref_f[:, 3]) <= 1.0 / net.n_species + 1e-6) >= 0.98
    qmis = np.mean(np.abs(gf[:, 4:] - ref_f[:, 4:]) > 1e-4)
    assert qmis < 0.02, qmis
    lmis = np.mean(np.abs(gl - ref_l) > 1e-4)
    assert lmis < 0.02, lmis
    g.close()


def _bf16(x):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("margin", [0.0, 0.5])
def test_in_integrator_inference_matches_oracle(env, margin):
    """The network evaluation the integrator itself runs (shared-memory BF16
    weights, FP32 accumulation on CUDA cores, one row per zone group) and
    the proposal rule dt = clip(dt_prev e^(out - margin), dt_plain, 16
    dt_plain), then clipped to t_end, element by element against the
    oracle, from the integrator's own trace of every proposal."""
    torch, kn, learned = env
    rng = np.random.default_rng(11)
    p = M.init_params(11)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.1, p[k].shape)
    p["b3"][:] = 0.3  # proposals on both sides of the plain step
    mu = rng.normal(0, 1, 64).astype(np.float32)
    mu[:4] = (1.3, 18.0, -25.0, 0.5)
    sigma = np.full(64, 8.0, np.float32)
    mlp = kn.MLP()
    flat = kn.mlp_pack(p)
    mlp.set_params(flat, mu, sigma)
    pf = kn.mlp_unpack(flat)  # the FP32 values the GPU holds
    net = net150()
    z = profile_zones(net, 12, base_seed=77_000, t_end=1e-10)
    g = kn.Network(net)
    g.set_zones(z)
    dev = torch.device("cuda")
    cap = 200_000
    tf = torch.full((cap, 64), float("nan"), dtype=torch.float32, device=dev)
    to = torch.full((cap,), float("nan"), dtype=torch.float32, device=dev)
    td = torch.full((cap, 6), float("nan"), dtype=torch.float64, device=dev)
    tc = torch.zeros(1, dtype=torch.int64, device=dev)
    o = kn.Opts(precision=kn.PREC_MIXED, mlp=mlp, mlp_margin=margin, trace_features=tf.data_ptr(),
                trace_out=to.data_ptr(), trace_dt=td.data_ptr(), trace_capacity=cap, trace_count=tc.data_ptr())
    kn.integrate_batch([g], o)
    r = g.get()
    assert (r["status"] == 0).all()
    n = int(tc.item())
    assert 1000 < n <= cap, n
    feat = tf[:n].cpu().numpy()
    out = to[:n].cpu().numpy().astype(np.float64)
    d = td[:n].cpu().numpy()
    assert np.isfinite(feat).all() and np.isfinite(out).all()
    # (1) the network output, against the oracle on the BF16 operands the
    # integrator uses (inputs, weights and hidden activations rounded to BF16)
    inv = (np.float32(1.0) / sigma).astype(np.float32)
    xs = ((feat - mu) * inv).astype(np.float32)
    X = _bf16(xs)
    h1 = _bf16(np.maximum(X @ _bf16(pf["W1"]) + pf["b1"], 0))
    h2 = _bf16(np.maximum(h1 @ _bf16(pf["W2"]) + pf["b2"], 0))
    ref = (h2 @ pf["W3"])[:, 0] + pf["b3"][0]
    scale = max(1.0, np.max(np.abs(ref)))
    err = np.abs(out - ref)
    # equal up to FP32 summation order ...
    assert np.mean(err <= 1e-5 * scale) >= 0.98, np.mean(err <= 1e-5 * scale)
    # ... which can flip the BF16 rounding of a hidden activation by one BF16
    # spacing (at most 2^-7 of its value).  Per row, one flip in h1 moves the
    # output by at most 2^-7 |h1_k| sum_n |W2_kn w3_n|, one flip in h2 by
    # 2^-7 |h2_n w3_n|; the rows that differ must stay within twice the sum.
    w2w3 = np.abs(_bf16(pf["W2"])) @ np.abs(pf["W3"][:, 0])
    flip = 2.0 ** -7 * (np.max(np.abs(h1) * w2w3, axis=1) + np.max(np.abs(h2 * pf["W3"][:, 0]), axis=1))
    bad = err > 1e-5 * scale
    assert np.all(err[bad] <= 2.0 * flip[bad] + 1e-5 * scale), np.max(err[bad] / flip[bad])
    # and against the plain FP64 network on unrounded inputs (BF16 effects only)
    ref64, _ = M.forward(pf, xs.astype(np.float64))
    assert np.linalg.norm(out - ref64) <= 2e-2 * np.linalg.norm(ref64)
    # (2) the proposal rule: dt_prev e^min(out - margin, 20) (FP32 exponential)
    h_prev, dt_plain, raw, step, used, rem = d.T
    e = np.exp(np.minimum(out.astype(np.float32) - np.float32(margin), np.float32(20.0)).astype(np.float64))
    assert np.allclose(raw, h_prev * e, rtol=4e-7, atol=0)
    # then exactly: clip to [dt_plain, 16 dt_plain], then to t_end; a proposal
    # not above dt_plain leaves the plain attempt min(dt_plain, t_end - t).
    # The mixed form's update takes the step in FP32 (dt_plain is an FP32
    # value already), so the step taken is that choice rounded to FP32.
    prop = np.minimum(raw, 16.0 * dt_plain)
    want64 = np.where(raw > dt_plain, np.minimum(prop, rem), np.minimum(dt_plain, rem))
    want_used = (raw > dt_plain) & (want64 > dt_plain)
    want_step = want64.astype(np.float32).astype(np.float64)
    assert np.array_equal(dt_plain, dt_plain.astype(np.float32).astype(np.float64))
    assert np.array_equal(step, want_step)
    assert np.array_equal(used.astype(bool), want_used)
    assert want_used.any() and (~want_used).any()
    assert kn.batch_stats([g])["proposals_used"] <= int(want_used.sum())
    mlp.close()
    g.close()


def test_perfect_proposal_follows_the_label(env, oracle_mod):
    """follow_label: every state reached by an accepted step tries the
    label's step (the largest grid step before the first failing one),
    which passed the test from that very state, so no proposal of the run
    is rejected.  The run is the measured ceiling of a learned proposal."""
    torch, kn, learned = env
    net = net150()
    z = profile_zones(net, 16, base_seed=31_000, t_end=3e-11)
    g = kn.Network(net)
    dev = torch.device("cuda")
    res = {}
    for follow in (0, 1):
        g.set_zones(z)
        cap = 100_000
        feat = torch.empty((cap, 64), dtype=torch.float32, device=dev)
        lab = torch.empty(cap, dtype=torch.float32, device=dev)
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        kn.integrate_batch([g], kn.Opts(precision=kn.PREC_FP64, record_features=feat.data_ptr(),
                                        record_labels=lab.data_ptr(), record_capacity=cap,
                                        record_count=cnt.data_ptr(), follow_label=follow))
        r = g.get()
        res[follow] = (r, kn.batch_stats([g]))
        assert (r["status"] == 0).all() and np.array_equal(r["t"], z.t_end)
    plain, ceil = res[0], res[1]
    # the ceiling run takes the label's step wherever it beats the plain one,
    # and needs no more steps than the plain controller
    assert ceil[1]["proposals_used"] > 0
    assert ceil[0]["steps"].sum() <= plain[0]["steps"].sum()
    # same accuracy contract as the plain controller: the free-running tier
    ref = oracle_mod.Oracle(net).integrate_batch(z, threads=8)
    m = ref["Y"] > 1e-10
    assert np.max(np.abs(ceil[0]["Y"][m] - ref["Y"][m]) / ref["Y"][m]) < 10 * 0.05
    g.close()


def _train_small(torch, kn, learned, n_zones=48, epochs=3, capacity=400_000):
    net = net150()
    jobs = [(net, profile_zones(net, n_zones, base_seed=500_000, t_end=1e-10)),
            (chain_network(), profile_zones(chain_network(), 16, base_seed=600_000, t_end=1e-4))]
    feat, lab = learned.generate_records(jobs, capacity)
    assert feat.shape[0] > 10_000 and torch.isfinite(feat).all() and torch.isfinite(lab).all()
    mlp, hist = learned.train_network(feat, lab, epochs=epochs, batch=2048, lr=1e-3)
    return mlp, hist


def test_learned_mode_is_judged_by_the_plain_test(env, oracle_mod):
    torch, kn, learned = env
    mlp, hist = _train_small(torch, kn, learned)
    assert hist[-1] < hist[0]
    net = net150()
    z = profile_zones(net, 24, base_seed=900_000, t_end=1e-10)
    g = kn.Network(net)
    g.set_zones(z)
    # margin 0: the raw proposal, so the learned path is exercised
    kn.integrate_batch([g], kn.Opts(precision=kn.PREC_MIXED, mlp=mlp, mlp_margin=0.0))
    r = g.get()
    st = kn.batch_stats([g])
    assert (r["status"] == 0).all() and np.array_equal(r["t"], z.t_end)
    assert st["proposals_used"] > 0
    ref = oracle_mod.Oracle(net).integrate_batch(z, threads=8)
    for i in range(z.n_zones):
        m = ref["Y"][i] > 1e-10
        assert np.max(np.abs(r["Y"][i][m] - ref["Y"][i][m]) / ref["Y"][i][m]) < 10 * 0.05
    drift = np.abs((r["Y"] * net.A).sum(1) - 1)
    assert (drift <= (r["steps"] + r["rejects"]) * 1e-6).all()
    mlp.close()


def test_learned_gain_at_equal_accuracy(env, oracle_mod, capsys):
    """Trained on the integrator's records from training zones; evaluated on
    fresh-seed zones.  Reports accepted steps, attempts and time of the plain
    and learned controllers and their end-state errors against an oracle run
    at 10x tighter tolerances."""
    torch, kn, learned = env
    mlp, hist = _train_small(torch, kn, learned, n_zones=128, epochs=4, capacity=2_000_000)
    net = net150()
    Z = 512
    z = profile_zones(net, Z, base_seed=900_000, t_end=1e-9)
    g = kn.Network(net)
    res = {}
    for name, o in (("plain", kn.Opts(precision=kn.PREC_MIXED)),
                    ("learned", kn.Opts(precision=kn.PREC_MIXED, mlp=mlp))):
        g.set_zones(z)
        kn.integrate_batch([g], o)
        torch.cuda.synchronize()
        g.set_zones(z)
        t0 = time.perf_counter()
        kn.integrate_batch([g], o)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        r = g.get()
        st = kn.batch_stats([g])
        assert (r["status"] == 0).all()
        res[name] = dict(time=el, steps=int(r["steps"].sum()), attempts=int(r["steps"].sum() + r["rejects"].sum()),
                         props=st["proposals_used"], Y=r["Y"])
    # accuracy against a tighter oracle run on a sample of zones
    pick = np.linspace(0, Z - 1, 8).astype(int)
    tight = oracle_mod.Oracle(net).integrate_batch(
        z.subset(pick), oracle_mod.OracleOpts(eps_r=0.005, eps_c=1e-7), threads=8)
    for name in res:
        errs = []
        for a, i in enumerate(pick):
            m = tight["Y"][a] > 1e-10
            errs.append(np.median(np.abs(res[name]["Y"][i][m] - tight["Y"][a][m]) / tight["Y"][a][m]))
        res[name]["err"] = float(np.median(errs))
    p, l = res["plain"], res["learned"]
    with capsys.disabled():
        print(f"\n[learned-dt gain] train loss {hist[0]:.4f} -> {hist[-1]:.4f}; "
              f"plain: {p['steps']} steps, {p['attempts']} attempts, {p['time']:.3f}s, err {p['err']:.3e}; "
              f"learned: {l['steps']} steps ({l['steps'] / p['steps']:.3f}x), {l['attempts']} attempts "
              f"({l['attempts'] / p['attempts']:.3f}x), {l['time']:.3f}s ({p['time'] / l['time']:.3f}x speed), "
              f"proposals used {l['props']}, err {l['err']:.3e}")
    # equal accuracy: the learned controller's error is not materially worse
    assert l["err"] <= 1.5 * p["err"] + 1e-3
    mlp.close()
