"""GPU checks of the network-size sweep (the single-network scaling study).

Every sweep network, one zone at the sweep's constant T9 = 7, rho = 1e8, runs
through the integrator against the oracle from 1e-12 to 3e-11 s (1.3k - 15k
steps at these hot conditions; the 16-species chain to 1e-6 s), in the
free-running tier: step counts within 2 % in FP64 and 10 % in the mixed form
(some networks reject often and a discontinuous decision can fall the other
way), and equal accuracy -- the GPU's end-state error against an oracle run
at 10x tighter tolerances no worse than the default oracle's own -- plus, where
that own error is below eps_r, the end state within 10 eps_r of the oracle's.
The sweep's GPU timing helper returns a positive per-step time for the
smallest and largest sizes.
"""
import numpy as np
import pytest

from kn_inputs import SWEEP_SIZES, constant_zones, sweep_network

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kn():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_5826_gb300 import build, kn
    build.build()
    return kn


@pytest.mark.parametrize("n", SWEEP_SIZES)
def test_sweep_network_matches_oracle(kn, oracle_mod, n):
    net = sweep_network(n)
    z = constant_zones(net, 1, T9=7.0, rho=1e8, t_end=3e-11 if n > 16 else 1e-6)
    orc = oracle_mod.Oracle(net)
    ref = orc.integrate(z, 0)
    tight = orc.integrate(z, 0, oracle_mod.OracleOpts(eps_r=0.005, eps_c=1e-7))
    mt = tight["Y"] > 1e-10
    e_orc = np.max(np.abs(ref["Y"][mt] - tight["Y"][mt]) / tight["Y"][mt])
    for prec in (kn.PREC_FP64, kn.PREC_MIXED):
        g = kn.Network(net)
        g.set_zones(z)
        kn.integrate_batch([g], kn.Opts(precision=prec))
        r = g.get()
        g.close()
        assert r["status"][0] == 0 and r["t"][0] == z.t_end[0]
        tol = 0.02 if prec == kn.PREC_FP64 else 0.10
        assert abs(int(r["steps"][0]) - ref["steps"]) <= max(2, tol * ref["steps"])
        e_gpu = np.max(np.abs(r["Y"][0][mt] - tight["Y"][mt]) / tight["Y"][mt])
        assert e_gpu <= 1.5 * e_orc + 0.05, (n, prec, e_gpu, e_orc)
        if e_orc < 0.05:
            m = ref["Y"] > 1e-10
            assert np.max(np.abs(r["Y"][0][m] - ref["Y"][m]) / ref["Y"][m]) < 10 * 0.05


def test_sweep_timing_helper(kn):
    from paper_1409_5826_gb300 import size_sweep
    for n in (SWEEP_SIZES[0], SWEEP_SIZES[-1]):
        t = size_sweep.single_zone_step_time(sweep_network(n), steps=200)
        assert t is not None and t["s_per_step"] > 0 and t["attempts"] >= 200
