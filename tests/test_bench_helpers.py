"""Host-side arithmetic of bench.py (no GPU): the per-zone tail statistics
from timer stamps, and the roofline byte and flop counts against values
worked by hand for a tiny network."""
import numpy as np

import bench
from kn_inputs import custom_network


def test_tail_stats_hand_worked():
    # four zones: fetched at 0, 0, 5, 7 ms and written back at 10, 4, 6, 9 ms
    ns = np.array([[0, 10], [0, 4], [5, 6], [7, 9]], dtype=np.int64) * 1_000_000 + 123
    steps = np.array([1000, 400, 100, 200])
    t = bench.tail_stats(ns, steps, groups=2)
    assert t["span_ms"] == 10.0
    assert t["queue_drained_ms"] == 7.0 and t["tail_ms"] == 3.0
    assert t["longest_zone"] == {"ms": 10.0, "accepted_steps": 1000, "fetched_at_ms": 0.0, "us_per_step": 10.0}
    # busy time 10 + 4 + 1 + 2 = 17 ms over 2 groups x 10 ms
    assert abs(t["group_occupancy"] - 0.85) < 1e-12
    assert t["finish_ms_p50_p90_p99_max"][-1] == 10.0


def test_roofline_counts_hand_worked():
    # a + b -> c (2-body), c -> a + b (1-body): R = 2, S_r = 3, S_p = 3, N = 3
    net = custom_network([1.0, 1.0, 2.0], [((0, 1), (2,)), ((2,), (0, 1))], [0.0, 0.0], [0.0, 0.0])
    s_r, s_p = net.slot_counts()
    assert (s_r, s_p) == (3, 3)
    # plan's figure per accepted step: 4 S_r + 4 (S_r + R) + 2 (S_r + S_p) + 4 S_p = 12 + 20 + 12 + 12
    assert bench.algorithmic_smem_bytes(net, 10) == 10 * 56
    # fuller count: 12 R + 8 S_r + 6 (S_r + S_p) + 8 N per step, 28 N per attempt
    assert bench.full_smem_bytes(net, 10, 5) == 10 * (24 + 24 + 36 + 24) + 15 * 84
    # FP64 flops: rates 5 R + fluxes 3 (2-body) + 1 (1-body) + gathers 6 per step, 11 N per attempt
    assert bench.algorithmic_flops(net, 10, 5) == 10 * (10 + 4 + 6) + 15 * 33
    assert bench.update_fp64_flops(net, 15) == 15 * 33


def test_qss_roofline_counts_hand_worked():
    # the same network: a QSS attempt adds the predicted state's rates, fluxes
    # and gathers (20 FP64 operations, as per accepted step) and 49 N = 147
    net = custom_network([1.0, 1.0, 2.0], [((0, 1), (2,)), ((2,), (0, 1))], [0.0, 0.0], [0.0, 0.0])
    assert bench.algorithmic_flops_qss(net, 10, 5) == 10 * 20 + 15 * (20 + 147)
    # shared memory: the plan's 56 B per accepted step, and again per attempt
    clk = {"sm_mhz": 1000.0}
    r = bench.smem_roofline([(net, 10, 5)], 1.0, clk, 1, qss=True)
    assert r["algorithmic_smem_bytes_per_launch"] == 10 * 56 + 15 * 56
    # fuller count: the flux and gather part (108 B) again per attempt, the
    # update (84 B per attempt) once
    assert r["full_count_smem_bytes_per_launch"] == 10 * 108 + 15 * 84 + 15 * 108


def test_reference_arm_line_keeps_the_contract():
    """`bench.py --impl reference` (the oracle on a bounded sample, CPU only)
    prints one JSON line with the contract's keys, on a short interval."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--t-end", "3e-12"], cwd=root, capture_output=True, text=True,
                         timeout=600, check=True).stdout.strip().splitlines()
    assert len(out) == 1
    d = json.loads(out[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "zone-steps/s" and d["config"]["workload"].endswith("3e-12 s")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "sample" in d["cpu_baseline"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_committed_profile_lines_parse():
    """The committed summary of the headline kernel carries both machine-readable
    lines bench.py reads (DRAM bytes per launch; issue and LSU activity)."""
    t = bench._profile_line("integrate_kernel_mixed_1216x150_full.md")
    i = bench._profile_issue_line("integrate_kernel_mixed_1216x150_full.md")
    assert t is not None and t[1] == 1216 and t[0] > 0
    assert i is not None and 0.0 < i[0] <= 100.0 and 0.0 < i[1] <= 100.0
    assert len(t[2]) == len(i[2]) == 64
