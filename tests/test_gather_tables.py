"""Host-only checks of the integrator's gather tables (no device needed).

kn_check_gather_tables builds the sliced gather list that sums F+_i and k_i
(Eq. 1; the species-reaction maps of Sec. 10 item (2)) for a network at a
precision and zone-group size, and verifies it on the host: every index in
range, split rows in consecutive lanes of a flagged slice, and the gather run
with V[v] = v + 1 giving every row's sum exactly once.  Here it runs over the
benchmark networks at every group size the tiler considers, and over random
tiny networks (including species no reaction touches and rows far longer than
the others), in both precisions.
"""
import numpy as np
import pytest

from kn_inputs import SWEEP_SIZES, chain_network, net150, net365, random_tiny_network, sweep_network


@pytest.fixture(scope="module")
def kn():
    from paper_1409_5826_gb300 import build, kn
    build.build()
    return kn


@pytest.mark.parametrize("which", ["chain", "net150", "net365"])
def test_benchmark_networks(kn, which):
    net = {"chain": chain_network, "net150": net150, "net365": net365}[which]()
    terms = sum(net.slot_counts())
    for prec in (kn.PREC_MIXED, kn.PREC_FP64, kn.PREC_MIXED_FP64):
        for G in (32, 64, 128, 160, 192, 256, 384, 512, 1024):
            st = kn.check_gather_tables(net, prec, G)
            # the longest warp sums at least its share of the terms
            assert st["warp_terms_per_lane"] * 32 * (G // 32) >= terms
            assert st["piece_cap"] >= 1 and st["slices"] >= 1


@pytest.mark.parametrize("n", SWEEP_SIZES)
def test_sweep_networks(kn, n):
    net = sweep_network(n)
    for prec in (kn.PREC_MIXED, kn.PREC_FP64):
        for G in (64, 128, 256, 512):
            kn.check_gather_tables(net, prec, G)


def test_random_networks(kn):
    for seed in range(60):
        net = random_tiny_network(3 + seed % 20, 2 + (7 * seed) % 40, seed)
        for prec in (kn.PREC_MIXED, kn.PREC_FP64, kn.PREC_MIXED_FP64):
            for G in (32, 64, 96):
                kn.check_gather_tables(net, prec, G)


def test_bad_arguments(kn):
    net = chain_network()
    for prec, G in ((3, 64), (kn.PREC_MIXED, 48), (kn.PREC_MIXED, 0), (kn.PREC_MIXED, 2048)):
        with pytest.raises(kn.KnError) as e:
            kn.check_gather_tables(net, prec, G)
        assert e.value.code == kn.KN_ERR_INVALID_ARG
