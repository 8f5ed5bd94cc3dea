"""Benchmark: batched explicit asymptotic integration on GB300.

Workload: 4096 zones of the synthetic 150-species / 1604-reaction network,
each with its own T9(t) = T0 exp(-t/tau), rho(t) = rho0 exp(-3t/tau) profile
(T0 ~ U[2,7], rho0 ~ logU[1e7,1e9], tau ~ logU[0.1,1] s), integrated from
t = 1e-12 s to 1e-9 s.  One step = one pass of the whole hot path over the
batch: load the zones' conditions from device-resident inputs, then the
persistent integrator (rates, fluxes, gathers, kappa-switched update, accept
test, dt control) until every zone reaches t_end.

Prints ONE JSON line (rank 0).  value = accepted zone-steps per second over
all ranks; zones_per_s alongside.  Beside the headline (the mixed form), each
other form is timed the same way -- warm-up steps, CUDA events on the
launching stream around each batch, the L2 flushed between batches, clocks
sampled during the timed batches -- and carries its own roofline: the FP64
form, the mixed form with the FP64 update, the mixed form with the learned
proposal, the uneven-size batch (16/48 : 150/1604 : 365/4400 = 1:2:1), the
perfect-proposal run that bounds any learned proposal, and the learned
network's training kernels.  --impl reference times the CPU FP64 oracle
instead (bounded sample of the same workload on the host cores).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "zone-steps/s and zones/s to t_end, 150sp/1604rx batch; learned-Δt vs plain"
T_END = 1e-9
N_ZONES = 4096
WORKLOAD = "4096 zones x 150sp/1604rx, T9/rho profiles, t 1e-12 -> 1e-9 s"


def workload_name(args):
    """The workload's name: the default batch's, or one built from --zones and --t-end."""
    if (args.zones, args.t_end) == (N_ZONES, T_END):
        return WORKLOAD
    return f"{args.zones} zones x 150sp/1604rx, T9/rho profiles, t 1e-12 -> {args.t_end:g} s"
# the uneven-size batch: 2048 zones, 1:2:1, the chain over its own interval
MIXED_ZONES = 2048


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="mixed", choices=["mixed", "mixed_fp64", "fp64", "qss_fp64", "qss_mixed"])
    ap.add_argument("--zones", type=int, default=N_ZONES)
    ap.add_argument("--t-end", type=float, default=T_END, help="integration end time (s)")
    ap.add_argument("--strong", action="store_true",
                    help="under torchrun: split one batch of --zones zones over the ranks, balanced by predicted "
                         "cost (strong scaling), instead of --zones zones per rank (weak scaling)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baselines")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP64 and learned-dt side measurements")
    ap.add_argument("--tpz", type=int, default=0)
    ap.add_argument("--tpc", type=int, default=0)
    ap.add_argument("--mlp-train", action="store_true",
                    help="instead of the batch benchmark: time the learned network's training kernels alone "
                         "(fused forward + backward per 64-row tile, gradient reduction, Adam) and print that line")
    ap.add_argument("--sweep", action="store_true",
                    help="instead of the batch benchmark: time one integration step of a single network "
                         "against its size (GPU, CPU oracle, CPU backward Euler) and print that table")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
                "power_w_max": float(max(power)), "reasons": sorted(reasons)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def algorithmic_flops(net, steps, rejects):
    """Algorithmic FP64 operations of the FP64 form per batch, counting a
    multiply or add as 1, an FMA as 2 and each exp/div as 1, with sentinel
    multiplications by 1 excluded:
      rates  5 per reaction per accepted step (2 FMA-equivalents + exp)
      fluxes+partials  1 / 3 / 7 per 1- / 2- / 3-body reaction per accepted step
      gathers  1 per product slot and reactant slot per accepted step
      update+test  11 per species per attempt (accepted or rejected)."""
    nr = net.n_reac
    R = net.n_reactions
    s_r, s_p = net.slot_counts()
    per_rx = np.where(nr == 1, 1, np.where(nr == 2, 3, 7)).sum()
    return float(steps * (5 * R + per_rx + s_r + s_p) + (steps + rejects) * 11 * net.n_species)


def algorithmic_flops_qss(net, steps, rejects):
    """Algorithmic FP64 operations of the alpha-QSS form per batch, counted as
    in algorithmic_flops: per accepted step the new state's rates, fluxes and
    gathers; per attempt the predicted state's rates, fluxes and gathers again,
    and 49 per species (alpha 11 twice; the predictor 8 more; the corrector 13
    more; the conservation sum and the relative test 6)."""
    nr = net.n_reac
    R = net.n_reactions
    s_r, s_p = net.slot_counts()
    per_state = 5 * R + np.where(nr == 1, 1, np.where(nr == 2, 3, 7)).sum() + s_r + s_p
    return float(steps * per_state + (steps + rejects) * (per_state + 49 * net.n_species))


def algorithmic_smem_bytes(net, steps):
    """The per-zone-step shared-memory figure of the measurement plan, in the
    FP32 widths of the mixed form, times the accepted steps of the batch:
    abundance reads 4 S_r, partial and flux writes 4 (S_r + R), 16-bit gather
    indices 2 (S_r + S_p) and flux reads of the F+ gathers 4 S_p."""
    R = net.n_reactions
    s_r, s_p = net.slot_counts()
    return float(steps * (4 * s_r + 4 * (s_r + R) + 2 * (s_r + s_p) + 4 * s_p))


def full_smem_bytes(net, steps, rejects):
    """A fuller count, for context: every value the step reads or writes once,
    in the width the mixed form keeps it.
      flux pass, per accepted step: per reaction the packed reactant ids (4 B),
        the cached rate (4 B) and the flux store (4 B); per reactant slot the
        abundance read (4 B) and the partial store (4 B):  12 R + 8 S_r
      gathers, per accepted step: per term a 16-bit index and a 4 B value, per
        row one 4 B store:  6 (S_r + S_p) + 8 N
      update and test, per attempt: per species the abundance pair, F+, k and
        A (20 B) read and the new pair (8 B) written:  28 N"""
    R = net.n_reactions
    s_r, s_p = net.slot_counts()
    N = net.n_species
    return float(steps * (12 * R + 8 * s_r + 6 * (s_r + s_p) + 8 * N) + (steps + rejects) * 28 * N)


def _profile_line(name):
    """The machine-readable line of a committed ncu summary:
    `traffic: dram_bytes=<B> zones=<Z> sources_sha256=<H>`; (bytes, zones, hash) or None."""
    import re
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    m = re.search(r"traffic: dram_bytes=(\d+) zones=(\d+) sources_sha256=([0-9a-f]+)", open(path).read())
    return (int(m.group(1)), int(m.group(2)), m.group(3)) if m else None


def _profile_issue_line(name):
    """The issue line of a committed ncu summary:
    `issue: active_pct=<P> lsu_pct=<Q> sources_sha256=<H>`; (P, Q, hash) or None."""
    import re
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    m = re.search(r"issue: active_pct=([0-9.]+) lsu_pct=([0-9.]+) sources_sha256=([0-9a-f]+)", open(path).read())
    return (float(m.group(1)), float(m.group(2)), m.group(3)) if m else None


def kernel_sources_sha256():
    """Hash of the code that defines the integrator kernel and its tables,
    with comments and blank lines removed (launch, tiling and autotuner code,
    and comments, do not change a launch's traffic)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("kn_integrate.cu", "kn_internal.h", "kn_tables.cu"):
        txt = open(os.path.join(ROOT, "paper_1409_5826_gb300", "csrc", f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        h.update("\n".join(ln.strip() for ln in txt.splitlines() if ln.strip()).encode())
    return h.hexdigest()


def _n_sms():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def run_reference(args, rank, world):
    """CPU FP64 oracle on a bounded sample of the same workload."""
    if rank != 0:
        return
    import oracle
    from kn_inputs import net150, profile_zones
    net = net150()
    orc = oracle.Oracle(net)
    zones = profile_zones(net, args.zones, t_end=args.t_end)
    threads = os.cpu_count() or 1
    pick = np.linspace(0, args.zones - 1, 24).astype(int)
    sub = zones.subset(pick)
    for _ in range(args.warmup):
        orc.integrate_batch(zones.subset(pick[:threads]), threads=threads)
    tot_steps = tot_zones = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = orc.integrate_batch(sub, threads=threads)
        tot_steps += int(r["steps"].sum())
        tot_zones += int((r["status"] == 0).sum())
    el = time.perf_counter() - t0
    v = tot_steps / el
    line = {"metric": METRIC, "value": v, "unit": "zone-steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "zones_per_s": tot_zones / el,
            "config": {"workload": workload_name(args), "zones": args.zones, "sample_zones": len(pick)},
            "cpu_baseline": {"value": v, "unit": "zone-steps/s", "cores": threads, "kind": "oracle",
                             "sample": f"{len(pick)} of the {args.zones} zones (evenly spaced), each step"},
            "e2e": {"value": v, "unit": "zone-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baselines(net, zones):
    """Oracle (explicit) and dense-LU backward Euler on bounded samples."""
    import oracle
    orc = oracle.Oracle(net)
    threads = os.cpu_count() or 1
    pick = np.linspace(0, zones.n_zones - 1, 24).astype(int)
    t0 = time.perf_counter()
    r = orc.integrate_batch(zones.subset(pick), threads=threads)
    el = time.perf_counter() - t0
    exp = {"value": float(r["steps"].sum() / el), "unit": "zone-steps/s", "cores": threads, "kind": "oracle",
           "sample": f"{len(pick)} evenly spaced zones of the batch, FP64 oracle, one thread per zone",
           "zones_per_s": float((r["status"] == 0).sum() / el),
           "s_per_step_per_core": float(el * min(threads, len(pick)) / r["steps"].sum())}
    bpick = np.linspace(0, zones.n_zones - 1, min(threads, 8)).astype(int)
    t0 = time.perf_counter()
    b = orc.be_integrate_batch(zones.subset(bpick), max_iter=6, threads=threads)
    bel = time.perf_counter() - t0
    be = {"value": float(b["steps"].sum() / bel), "unit": "zone-steps/s", "cores": threads,
          "kind": "backward Euler, dense LU, Newton <= 6 iterations",
          "sample": f"{len(bpick)} evenly spaced zones of the batch",
          "zones_per_s": float((b["status"] == 0).sum() / bel),
          "s_per_step_per_core": float(bel * len(bpick) / max(1, b["steps"].sum()))}
    return exp, be


def size_sweep(args):
    """The single-network scaling study at constant T9 = 7, rho = 1e8: time per
    accepted step of one zone on the GPU (fastest one-group tiling), of the FP64
    oracle on one host core and of dense-LU backward Euler on one host core,
    plus the GPU batch throughput at each size.  One JSON line."""
    import oracle
    from kn_inputs import SWEEP_SIZES, constant_zones, sweep_network
    from paper_1409_5826_gb300 import build, size_sweep as sw
    build.build()
    rows = sw.run(SWEEP_SIZES, steps=2000, batch_zones=4096)
    for row in rows:
        net = sweep_network(row["n_species"])
        orc = oracle.Oracle(net)
        z = constant_zones(net, 1, T9=sw.T9, rho=sw.RHO, t_end=sw.T_END)
        t0 = time.perf_counter()
        r = orc.integrate(z, 0, oracle.OracleOpts(max_steps=2000))
        el = time.perf_counter() - t0
        row["cpu_oracle_explicit"] = {"s_per_step": el / max(1, r["steps"]), "steps": int(r["steps"]), "cores": 1}
        be_steps = 200 if net.n_species <= 64 else (50 if net.n_species <= 150 else 20)
        t0 = time.perf_counter()
        b = orc.be_integrate(z, 0, oracle.OracleOpts(max_steps=be_steps), max_iter=6)
        el = time.perf_counter() - t0
        row["cpu_backward_euler"] = {"s_per_step": el / max(1, b["steps"]), "steps": int(b["steps"]), "cores": 1,
                                     "kind": "dense LU, Newton <= 6 iterations"}
        g = row["gpu_single_zone"]["s_per_step"]
        row["explicit_cpu_over_gpu"] = row["cpu_oracle_explicit"]["s_per_step"] / g
        row["be_cpu_over_gpu"] = row["cpu_backward_euler"]["s_per_step"] / g
    print(json.dumps({"sweep": "time per integration step vs network size, one zone at T9 = 7, rho = 1e8",
                      "rows": rows}), flush=True)


def single_zone_configs():
    """The measurement plan's single-zone configurations at constant T9 = 3,
    rho = 1e8: the 16/48 chain and the 150/1604 network.  Time per accepted
    step of one zone on the GPU (FP64 and mixed forms, fastest one-group
    tiling), of the FP64 oracle on one host core and of dense-LU backward
    Euler on one host core."""
    import oracle
    from kn_inputs import chain_network, constant_zones, net150
    from paper_1409_5826_gb300 import kn, size_sweep as sw
    out = {}
    for name, net in (("chain16_48", chain_network()), ("net150_1604", net150())):
        row = {}
        for form, prec in (("fp64", kn.PREC_FP64), ("mixed", kn.PREC_MIXED)):
            t = sw.single_zone_step_time(net, steps=2000, precision=prec, T9=3.0, rho=1e8)
            row[f"gpu_{form}_s_per_step"] = t["s_per_step"]
            row[f"gpu_{form}_threads_per_zone"] = t["threads_per_zone"]
        orc = oracle.Oracle(net)
        z = constant_zones(net, 1, T9=3.0, rho=1e8, t_end=sw.T_END)
        t0 = time.perf_counter()
        r = orc.integrate(z, 0, oracle.OracleOpts(max_steps=2000))
        row["cpu_oracle_s_per_step"] = (time.perf_counter() - t0) / max(1, r["steps"])
        t0 = time.perf_counter()
        b = orc.be_integrate(z, 0, oracle.OracleOpts(max_steps=200 if net.n_species <= 64 else 30), max_iter=6)
        row["cpu_backward_euler_s_per_step"] = (time.perf_counter() - t0) / max(1, b["steps"])
        row["cores"] = 1
        out[name] = row
    out["conditions"] = "one zone, T9 = 3, rho = 1e8 constant, 2000 steps (backward Euler: 200 / 30)"
    return out


def _sm_clock_hz(clk):
    return (clk.get("sm_mhz") or 2070.0) * 1e6


def timed_batches(kn, nets, set_zones, opts, steps, warmup, stream, flush, zone_ns=None, barrier=None):
    """`warmup` untimed batches, then `steps` timed ones.  Each timed batch:
    the L2 flushed (untimed), then CUDA events on the launching stream around
    the zone upload and the integration.  nvidia-smi clocks are sampled
    during the timed batches.  zone_ns: a device [zones][2] int64 tensor that
    receives the per-zone fetch and write-back times of every batch (the last
    one is read back)."""
    import torch
    o = kn.Opts(**{**opts.__dict__, "zone_ns": zone_ns.data_ptr() if zone_ns is not None else 0})
    for _ in range(warmup):
        set_zones()
        kn.integrate_batch(nets, o, stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    if barrier:
        barrier()
    torch.cuda.synchronize()
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        set_zones()
        ev[i][1].record(stream)
        kn.integrate_batch(nets, o, stream)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    clk = clocks.stop()
    return {"step_ms": [a.elapsed_time(c) for a, b, c in ev], "kernel_ms": [b.elapsed_time(c) for a, b, c in ev],
            "clocks": clk, "stats": kn.batch_stats(nets, stream),
            "zone_ns": zone_ns.cpu().numpy() if zone_ns is not None else None}


def tail_stats(zone_ns, steps, groups):
    """From the per-zone timer stamps of one batch: the batch span, when the
    work queue drained (the last fetch), the time after that (the tail), the
    spread of zone finish times, the longest zone, and the mean occupancy of
    the zone groups."""
    ns = zone_ns.astype(np.float64)
    t0 = ns[:, 0].min()
    fetch = (ns[:, 0] - t0) / 1e6
    end = (ns[:, 1] - t0) / 1e6
    dur = end - fetch
    i = int(np.argmax(dur))
    span = float(end.max())
    return {"span_ms": span, "queue_drained_ms": float(fetch.max()), "tail_ms": float(span - fetch.max()),
            "finish_ms_p50_p90_p99_max": [float(np.percentile(end, q)) for q in (50, 90, 99, 100)],
            "longest_zone": {"ms": float(dur[i]), "accepted_steps": int(steps[i]), "fetched_at_ms": float(fetch[i]),
                             "us_per_step": float(dur[i] * 1e3 / max(1, steps[i]))},
            "group_occupancy": float(dur.sum() / (groups * span)) if groups else None}


def _mean(x):
    return float(np.mean(x))


def smem_roofline(parts, kms, clk, n_sms, qss=False):
    """Shared-memory roofline of the FP32-flux forms: the measurement plan's
    bytes per accepted zone-step (algorithmic_smem_bytes, FP32 widths) over
    the kernel time, against 128 B/clk/SM x SMs x the sampled SM clock.
    parts: [(network, accepted steps, rejects)].  qss: the QSS update, whose
    every attempt also runs the flux pass and the gathers of the predicted
    state (the same bytes again per attempt)."""
    peak = 128.0 * n_sms * _sm_clock_hz(clk) / 1e9
    b = sum(algorithmic_smem_bytes(n, st) + (algorithmic_smem_bytes(n, st + rj) if qss else 0.0)
            for n, st, rj in parts)
    bf = sum(full_smem_bytes(n, st, rj) + (full_smem_bytes(n, st + rj, 0) - 28 * n.n_species * (st + rj)
                                          if qss else 0.0)
             for n, st, rj in parts)
    return {"bound": "alu", "resource": "shared-memory bandwidth (SM-local)", "unit": "GB/s",
            "kernel": "integrate_kernel", "achieved": b / (kms / 1e3) / 1e9, "peak": peak,
            "frac": b / (kms / 1e3) / 1e9 / peak,
            "peak_source": "derived: 128 B/clk/SM x SMs x sampled SM clock",
            "algorithmic_smem_bytes_per_launch": b,
            "algorithmic_unit": "per accepted zone-step: 4 S_r + 4 (S_r + R) + 2 (S_r + S_p) + 4 S_p bytes",
            "full_count_smem_bytes_per_launch": bf, "full_count_frac": bf / (kms / 1e3) / 1e9 / peak,
            "kernel_ms": kms}


def fp64_roofline(flops, kms, fp64_peak, what):
    return {"bound": "alu", "resource": "FP64 pipe", "unit": "TFLOP/s", "kernel": "integrate_kernel",
            "achieved": flops / (kms / 1e3) / 1e12, "peak": fp64_peak, "frac": flops / (kms / 1e3) / 1e12 / fp64_peak,
            "peak_source": "measured FP64 DFMA throughput (kn_measure_fp64_peak)",
            "algorithmic_fp64_flops_per_launch": flops, "algorithmic_unit": what, "kernel_ms": kms,
            "nominal_fp64_tflops": 1.25}


def update_fp64_flops(net, attempts):
    """FP64 operations of the kappa-switched update, the conservation sum and
    the relative test: 11 per species per attempt (as in algorithmic_flops)."""
    return float(attempts * 11 * net.n_species)


def _form_line(tb, nets, zones_total, roof, extra=None):
    st = tb["stats"]
    kms = _mean(tb["kernel_ms"])
    out = {"zone_steps_per_s": st["steps"] / (kms / 1e3), "zones_per_s": st["zones_ok"] / (kms / 1e3),
           "ms_per_batch": _mean(tb["step_ms"]), "kernel_ms": kms, "kernel_ms_all": tb["kernel_ms"],
           "accepted_steps": st["steps"], "rejects": st["rejects"], "zones": zones_total,
           "zones_ok": st["zones_ok"], "clocks": tb["clocks"], "roofline": roof}
    if extra:
        out.update(extra)
    return out


def other_forms(kn, g, net, zones, dz, stream, flush, mixed_line, args):
    """Every other form on the same batch, timed like the headline (3 warm-up
    and 3 timed batches; the FP64 form, at ~10 s a batch, 1 + 2), each with
    its roofline and its end-state error against an oracle run at 10x
    tighter tolerances on 8 zones; then the perfect-proposal run, the
    uneven-size batch and the learned network's training kernels."""
    import torch
    import oracle
    from kn_inputs import chain_network, net365, profile_zones, mixed_assignment
    from paper_1409_5826_gb300 import learned
    out = {}
    n_sms = _n_sms()
    fp64_peak = kn.measure_fp64_peak(stream)
    pick = np.linspace(0, zones.n_zones - 1, 8).astype(int)
    tight = oracle.Oracle(net).integrate_batch(zones.subset(pick), oracle.OracleOpts(eps_r=0.005, eps_c=1e-7),
                                               threads=os.cpu_count() or 1)

    def err():
        Y = g.get(stream)["Y"]
        e = []
        for a, i in enumerate(pick):
            m = tight["Y"][a] > 1e-10
            e.append(np.median(np.abs(Y[i][m] - tight["Y"][a][m]) / tight["Y"][a][m]))
        return float(np.median(e))

    def set_main():
        g.set_zones(dz, stream)

    zns = torch.zeros((zones.n_zones, 2), dtype=torch.int64, device=torch.device("cuda", torch.cuda.current_device()))

    def tail_of(tb, tuned):
        groups = n_sms * (tuned["threads_per_cta"] // tuned["threads_per_zone"]) if tuned else None
        return tail_stats(tb["zone_ns"], g.get(stream)["steps"], groups)

    out["mixed"] = {"median_rel_err_vs_tight_oracle": err(), "see": "the headline value and roofline"}
    # the split the measurement plan names: FP32 rates, fluxes and Kahan
    # gathers; FP64 update, conservation sum and test
    g.set_zones(dz, stream)
    # whole-batch trials: steady-state trials rank this FP64-pipe-bound form's
    # tilings differently from the whole batch (measured: 4 x 160 against 2 x 160)
    tuned = kn.autotune([g], kn.Opts(precision=kn.PREC_MIXED_FP64), max_steps=0, stream=stream)
    tb = timed_batches(kn, [g], set_main, kn.Opts(precision=kn.PREC_MIXED_FP64, use_graph=1), 3, 3, stream, flush,
                       zns)
    kms = _mean(tb["kernel_ms"])
    st = tb["stats"]
    roof = fp64_roofline(update_fp64_flops(net, st["steps"] + st["rejects"]), kms, fp64_peak,
                         "11 FP64 operations per species per attempt (update, conservation sum, test)")
    roof["smem"] = smem_roofline([(net, st["steps"], st["rejects"])], kms, tb["clocks"], n_sms)
    out["mixed_fp64_update"] = _form_line(tb, [g], zones.n_zones, roof,
                                          {"median_rel_err_vs_tight_oracle": err(), "tiling": tuned,
                                           "tail": tail_of(tb, tuned)})
    # every step in FP64
    g.set_zones(dz, stream)
    tuned = kn.autotune([g], kn.Opts(precision=kn.PREC_FP64), max_steps=100, stream=stream)
    tb = timed_batches(kn, [g], set_main, kn.Opts(precision=kn.PREC_FP64, use_graph=1), 2, 1, stream, flush, zns)
    st = tb["stats"]
    roof = fp64_roofline(algorithmic_flops(net, st["steps"], st["rejects"]), _mean(tb["kernel_ms"]), fp64_peak,
                         "rates 5 R + fluxes 1/3/7 per 1/2/3-body reaction + gathers S_r + S_p per accepted step, "
                         "11 N per attempt")
    out["fp64"] = _form_line(tb, [g], zones.n_zones, roof, {"median_rel_err_vs_tight_oracle": err(), "tiling": tuned,
                                                            "tail": tail_of(tb, tuned)})
    # the alpha-QSS update in FP64 (Sec. 11's question: does QSS in place of
    # Eq. 3 integrate faster on the GPU?); the same accept test and controller
    g.set_zones(dz, stream)
    qo = dict(precision=kn.PREC_FP64, method=kn.METHOD_QSS)
    tuned = kn.autotune([g], kn.Opts(**qo), max_steps=100, stream=stream)
    tb = timed_batches(kn, [g], set_main, kn.Opts(**qo, use_graph=1), 1, 1, stream, flush, zns)
    st = tb["stats"]
    roof = fp64_roofline(algorithmic_flops_qss(net, st["steps"], st["rejects"]), _mean(tb["kernel_ms"]), fp64_peak,
                         "rates 5 R + fluxes 1/3/7 per 1/2/3-body reaction + gathers S_r + S_p per accepted step "
                         "and again per attempt (the predicted state), 49 N per attempt")
    out["qss_fp64"] = _form_line(tb, [g], zones.n_zones, roof, {"median_rel_err_vs_tight_oracle": err(),
                                                                "tiling": tuned, "tail": tail_of(tb, tuned)})
    out["qss_vs_asymptotic_fp64_zones_per_s"] = out["qss_fp64"]["zones_per_s"] / out["fp64"]["zones_per_s"]
    # the same in the mixed form, against the headline
    g.set_zones(dz, stream)
    qo = dict(precision=kn.PREC_MIXED, method=kn.METHOD_QSS)
    tuned = kn.autotune([g], kn.Opts(**qo), max_steps=300, stream=stream)
    tb = timed_batches(kn, [g], set_main, kn.Opts(**qo, use_graph=1), 3, 3, stream, flush, zns)
    st = tb["stats"]
    roof = smem_roofline([(net, st["steps"], st["rejects"])], _mean(tb["kernel_ms"]), tb["clocks"], n_sms,
                         qss=True)
    out["qss_mixed"] = _form_line(tb, [g], zones.n_zones, roof, {"median_rel_err_vs_tight_oracle": err(),
                                                                 "tiling": tuned, "tail": tail_of(tb, tuned)})
    out["qss_vs_asymptotic_mixed_zones_per_s"] = out["qss_mixed"]["zones_per_s"] / mixed_line["zones_per_s"]
    # the learned proposal: records from training zones, training on the GPU,
    # then the batch with the network proposing and the plain test judging
    t0 = time.perf_counter()
    jobs = [(net, profile_zones(net, 128, base_seed=500_000, t_end=T_END)),
            (chain_network(), profile_zones(chain_network(), 32, base_seed=600_000, t_end=1e-2))]
    feat, lab = learned.generate_records(jobs, 2_000_000, stream=stream)
    rec_s = time.perf_counter() - t0
    # untimed warm-up on a slice: the first use of torch's shuffle, gather and
    # reduction kernels in the process loads them (about 4 s on a fresh box)
    learned.train_network(feat[:65536], lab[:65536], epochs=1, batch=4096, stream=stream)[0].close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mlp, hist, train_kernel_s = learned.train_network(feat, lab, epochs=4, batch=4096, lr=1e-3, stream=stream,
                                                      time_kernels=True)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    g.set_zones(dz, stream)
    tuned = kn.autotune([g], kn.Opts(precision=kn.PREC_MIXED, mlp=mlp), max_steps=300, stream=stream)
    tb = timed_batches(kn, [g], set_main, kn.Opts(precision=kn.PREC_MIXED, mlp=mlp, use_graph=1), 3, 3, stream, flush,
                       zns)
    st = tb["stats"]
    kms = _mean(tb["kernel_ms"])
    roof = smem_roofline([(net, st["steps"], st["rejects"])], kms, tb["clocks"], n_sms)
    # the network evaluation on CUDA cores: 2 (64 128 + 128 128 + 128) flops
    # per proposal, one proposal per state reached by an accepted step
    mlp_flops = 2.0 * (64 * 128 + 128 * 128 + 128) * (st["steps"] - zones.n_zones)
    fp32_peak = 2.0 * 128 * n_sms * _sm_clock_hz(tb["clocks"]) / 1e12
    roof["mlp_inference"] = {"unit": "TFLOP/s", "flops_per_launch": mlp_flops,
                             "achieved_over_kernel_time": mlp_flops / (kms / 1e3) / 1e12, "peak": fp32_peak,
                             "peak_source": "derived: 128 FP32 FMA lanes/clk/SM x 2 x SMs x sampled clock"}
    out["mixed_learned"] = _form_line(tb, [g], zones.n_zones, roof, {
        "proposals_used": st["proposals_used"], "median_rel_err_vs_tight_oracle": err(), "tiling": tuned,
        "tail": tail_of(tb, tuned),
        "records": int(feat.shape[0]), "record_gen_s": rec_s, "train_s": train_s,
        "train_kernel_s": train_kernel_s, "train_loss_first_last": [hist[0], hist[-1]]})
    out["learned_vs_plain_mixed_zones_per_s"] = out["mixed_learned"]["zones_per_s"] / mixed_line["zones_per_s"]
    out["learned_mixed_vs_plain_fp64_zones_per_s"] = out["mixed_learned"]["zones_per_s"] / out["fp64"]["zones_per_s"]
    del feat, lab
    # the learned network's training kernels alone: fused forward + backward
    # and the Adam step on batches of 4096 records, back to back
    out["mlp_training_kernels"] = mlp_training_roofline(kn, mlp, stream)
    mlp.close()
    # the perfect proposal: every state reached by an accepted step tries the
    # step the records' label names (the largest grid step before the first
    # that fails), clipped like a learned proposal; what it saves bounds what
    # any learned proposal of this form can save
    out["perfect_proposal_ceiling"] = perfect_proposal(kn, g, dz, stream)
    # the uneven-size batch: 16/48 : 150/1604 : 365/4400 = 1:2:1 in one launch
    out["uneven_sizes"] = uneven_sizes(kn, stream, flush, n_sms, args)
    out["qss_chain"] = qss_chain(kn, stream, flush, fp64_peak)
    out["note"] = ("every form: warm-up batches, then timed batches with CUDA events on the launching stream, "
                   "L2 flushed between batches, clocks sampled; errors against an oracle run at eps_r 0.005, "
                   "eps_c 1e-7 on 8 zones of the batch")
    return out


def mlp_training_roofline(kn, mlp, stream, B=4096, batches=200):
    """CUDA-event time of `batches` training steps (kn_mlp_backward: the fused
    forward + backward tile kernel and the partial-gradient reduction; then
    kn_mlp_adam) on random records, against the BF16 tensor peak."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    gen = torch.Generator(device=dev)
    gen.manual_seed(3)
    feat = torch.randn((B, 64), generator=gen, device=dev, dtype=torch.float32)
    lab = torch.randn(B, generator=gen, device=dev, dtype=torch.float32)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    for _ in range(5):
        mlp.backward(feat, lab, loss, stream)
        mlp.adam(1e-6, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(batches):
        mlp.backward(feat, lab, loss, stream)
        mlp.adam(1e-6, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / batches
    # GEMM flops per step: forward 2 B (64 128 + 128 128); backward dZ1 2 B 128 128,
    # dW2 2 B 128 128, dW1 2 B 64 128
    flops = 2.0 * B * (64 * 128 + 128 * 128) + 2.0 * B * (128 * 128 + 128 * 128 + 64 * 128)
    peaks, src = _peaks()
    return {"batch": B, "us_per_training_step": us, "gemm_flops_per_step": flops,
            "achieved_tflops": flops / (us / 1e6) / 1e12, "peak_tflops": peaks["bf16_tflops"],
            "frac": flops / (us / 1e6) / 1e12 / peaks["bf16_tflops"],
            "peak_source": f"MEASURED_PEAKS.json bf16_tflops ({src}), dense BF16", "bound": "tensor",
            "launches_per_step": 3}


def perfect_proposal(kn, g, dz, stream):
    """Accepted steps and attempts of the plain controller and of the perfect
    proposal on the bench batch (mixed form; untimed: the label search runs
    the update up to 25 times per state)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    feat = torch.empty((1, 64), dtype=torch.float32, device=dev)
    lab = torch.empty(1, dtype=torch.float32, device=dev)
    res = {}
    for follow in (0, 1):
        cnt = torch.zeros(1, dtype=torch.int64, device=dev)
        g.set_zones(dz, stream)
        t0 = time.perf_counter()
        kn.integrate_batch([g], kn.Opts(precision=kn.PREC_MIXED, record_features=feat.data_ptr(),
                                        record_labels=lab.data_ptr(), record_capacity=0,
                                        record_count=cnt.data_ptr(), follow_label=follow), stream)
        torch.cuda.synchronize()
        st = kn.batch_stats([g], stream)
        res["perfect" if follow else "plain"] = {"accepted_steps": st["steps"], "rejects": st["rejects"],
                                                 "attempts": st["steps"] + st["rejects"],
                                                 "proposals_used": st["proposals_used"],
                                                 "wall_s": time.perf_counter() - t0}
    p, q = res["plain"], res["perfect"]
    res["steps_ratio"] = q["accepted_steps"] / p["accepted_steps"]
    res["attempts_ratio"] = q["attempts"] / p["attempts"]
    res["note"] = ("perfect: at every state the label's step (largest grid step dt_prev 2^(k/4) before the first "
                   "that fails), clipped to [dt_plain, 16 dt_plain]; attempts_ratio is the most a learned "
                   "proposal could save")
    return res


def qss_chain(kn, stream, flush, fp64_peak):
    """The alpha-QSS update against Eq. 3, in FP64 and in the mixed form, on
    4096 zones of the 16-species chain with profiles over 1e-12 -> 1e-2 s
    (where the oracle takes 3-4x fewer steps with QSS), each with its
    roofline and its end-state error against a 10x-tighter Eq. 3 oracle run
    on 8 zones."""
    import torch
    import oracle
    from kn_inputs import chain_network, profile_zones
    net = chain_network()
    zones = profile_zones(net, 4096, base_seed=700_000, t_end=1e-2)
    dev = torch.device("cuda", torch.cuda.current_device())
    names = ("Y0", "T0", "rho0", "tau", "t_start", "t_end", "dt_trial")
    dz = {k: torch.from_numpy(np.ascontiguousarray(getattr(zones, k))).to(dev) for k in names}
    g = kn.Network(net)
    pick = np.linspace(0, zones.n_zones - 1, 8).astype(int)
    tight = oracle.Oracle(net).integrate_batch(zones.subset(pick), oracle.OracleOpts(eps_r=0.005, eps_c=1e-7),
                                               threads=os.cpu_count() or 1)

    def set_main():
        g.set_zones(dz, stream)

    out = {"workload": "4096 zones x 16sp/48rx chain, T9/rho profiles, t 1e-12 -> 1e-2 s"}
    n_sms = _n_sms()
    for name, prec, method, count in (("asymptotic_fp64", kn.PREC_FP64, kn.METHOD_ASYMPTOTIC, algorithmic_flops),
                                      ("qss_fp64", kn.PREC_FP64, kn.METHOD_QSS, algorithmic_flops_qss),
                                      ("asymptotic_mixed", kn.PREC_MIXED, kn.METHOD_ASYMPTOTIC, None),
                                      ("qss_mixed", kn.PREC_MIXED, kn.METHOD_QSS, None)):
        o = dict(precision=prec, method=method)
        set_main()
        tuned = kn.autotune([g], kn.Opts(**o), max_steps=3000, stream=stream)
        tb = timed_batches(kn, [g], set_main, kn.Opts(**o, use_graph=1), 3, 3, stream, flush)
        st = tb["stats"]
        kms = _mean(tb["kernel_ms"])
        if count:
            roof = fp64_roofline(count(net, st["steps"], st["rejects"]), kms, fp64_peak,
                                 "as the 150-species forms' FP64 counts")
        else:
            roof = smem_roofline([(net, st["steps"], st["rejects"])], kms, tb["clocks"], n_sms,
                                 qss=method == kn.METHOD_QSS)
        Y = g.get(stream)["Y"]
        e = [np.median(np.abs(Y[i][m] - tight["Y"][a][m]) / tight["Y"][a][m])
             for a, i in enumerate(pick) for m in [tight["Y"][a] > 1e-10]]
        out[name] = _form_line(tb, [g], zones.n_zones, roof, {"median_rel_err_vs_tight_oracle": float(np.median(e)),
                                                              "tiling": tuned})
    out["qss_vs_asymptotic_fp64_zones_per_s"] = out["qss_fp64"]["zones_per_s"] / out["asymptotic_fp64"]["zones_per_s"]
    out["qss_vs_asymptotic_mixed_zones_per_s"] = (out["qss_mixed"]["zones_per_s"] /
                                                  out["asymptotic_mixed"]["zones_per_s"])
    return out


def uneven_sizes(kn, stream, flush, n_sms, args):
    """2048 zones of the 16/48, 150/1604 and 365/4400 networks in the ratio
    1:2:1 (shuffled assignment, config-3 profiles; the chain over 1e-12 ->
    1e-2 s, the others over 1e-12 -> 1e-9 s: kn_inputs.uneven_batch), all in
    one persistent launch with the autotuned tiling."""
    import torch
    from kn_inputs import UNEVEN_T_END, uneven_batch
    dev = torch.device("cuda", torch.cuda.current_device())
    names = ("Y0", "T0", "rho0", "tau", "t_start", "t_end", "dt_trial")
    gs, dzs, counts, nets = [], [], {}, {}
    for name, net, z, idx in uneven_batch(MIXED_ZONES):
        g = kn.Network(net)
        d = {n: torch.from_numpy(np.ascontiguousarray(getattr(z, n))).to(dev) for n in names}
        gs.append(g)
        dzs.append(d)
        counts[name] = int(len(idx))
        nets[name] = net

    def set_all():
        for g, d in zip(gs, dzs):
            g.set_zones(d, stream)

    set_all()
    tuned = kn.autotune(gs, kn.Opts(precision=kn.PREC_MIXED), max_steps=0, stream=stream)
    zns = torch.zeros((MIXED_ZONES, 2), dtype=torch.int64, device=dev)
    tb = timed_batches(kn, gs, set_all, kn.Opts(precision=kn.PREC_MIXED, use_graph=1), 3, 3, stream, flush, zns)
    kms = _mean(tb["kernel_ms"])
    per, parts, steps_all = {}, [], []
    for (name, net), g in zip(nets.items(), gs):
        st = kn.batch_stats([g], stream)
        r = g.get(stream)
        steps_all.append(r["steps"])
        per[name] = {"zones": counts[name], "zones_ok": st["zones_ok"], "accepted_steps": st["steps"],
                     "rejects": st["rejects"], "zones_per_s": st["zones_ok"] / (kms / 1e3),
                     "zone_steps_per_s": st["steps"] / (kms / 1e3), "t_end": UNEVEN_T_END[name]}
        parts.append((net, st["steps"], st["rejects"]))
    roof = smem_roofline(parts, kms, tb["clocks"], n_sms)
    line = _form_line(tb, gs, MIXED_ZONES, roof, {"per_network": per, "tiling": tuned})
    line["tail"] = tail_stats(tb["zone_ns"], np.concatenate(steps_all), None)
    for g in gs:
        g.close()
    return line


def main():
    args = _args()
    rank, world, local = _dist()
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, rank, world)
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.sweep:
        if rank == 0:
            size_sweep(args)
        return
    if args.mlp_train:
        if rank == 0:
            import torch
            from paper_1409_5826_gb300 import build, kn, learned
            build.build()
            mlp = kn.MLP()
            mlp.set_params(learned.init_params(0), np.zeros(64, np.float32), np.ones(64, np.float32))
            print(json.dumps({"mlp_training_kernels": mlp_training_roofline(kn, mlp, torch.cuda.current_stream(),
                                                                            batches=args.steps)}), flush=True)
            mlp.close()
        return
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from kn_inputs import net150, profile_zones
    from paper_1409_5826_gb300 import build, kn
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    build.build()
    net = net150()
    from paper_1409_5826_gb300 import shard
    if args.strong:
        # strong scaling: one batch, split over the ranks balanced by predicted cost
        whole = profile_zones(net, args.zones, t_end=args.t_end)
        zones = whole.subset(shard.balanced_partition(shard.cost_key(net, whole), world)[rank])
    else:
        # weak scaling: each rank integrates its own slice of the global batch
        zones = profile_zones(net, args.zones, base_seed=shard.zone_seed_base(rank, world, args.zones),
                              t_end=args.t_end)
    dev = torch.device("cuda", local)
    names = ("Y0", "T0", "rho0", "tau", "t_start", "t_end", "dt_trial")
    dz = {k: torch.from_numpy(np.ascontiguousarray(getattr(zones, k))).to(dev) for k in names}
    g = kn.Network(net)
    prec = {"mixed": kn.PREC_MIXED, "mixed_fp64": kn.PREC_MIXED_FP64, "fp64": kn.PREC_FP64,
            "qss_fp64": kn.PREC_FP64, "qss_mixed": kn.PREC_MIXED}[args.form]
    method = kn.METHOD_QSS if args.form.startswith("qss") else kn.METHOD_ASYMPTOTIC
    stream = torch.cuda.current_stream()
    tuned = None
    if not (args.tpz or args.tpc):
        # the project's autotuner picks the tiling on this batch (untimed
        # set-up; whole-batch trials, since the batch's tail matters here)
        g.set_zones(dz, stream)
        tuned = kn.autotune([g], kn.Opts(precision=prec, method=method), max_steps=0, stream=stream)
    opts = kn.Opts(precision=prec, method=method, use_graph=1, threads_per_zone=args.tpz, threads_per_cta=args.tpc)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    def set_main():
        g.set_zones(dz, stream)

    zns = torch.zeros((zones.n_zones, 2), dtype=torch.int64, device=dev)
    tb = timed_batches(kn, [g], set_main, opts, args.steps, max(3, args.warmup), stream, flush, zns,
                       barrier=dist.barrier if world > 1 else None)
    clk = tb["clocks"]
    ms = float(np.sum(tb["step_ms"]))
    st = tb["stats"]
    steps_per_batch = st["steps"]
    zones_ok = st["zones_ok"]
    zone_steps = g.get(stream)["steps"]
    ms, steps_all, zones_all = shard.aggregate(ms, steps_per_batch, zones_ok, device=dev)
    value = steps_all * args.steps / (ms / 1e3)

    # end to end through the public API with pinned host buffers
    pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(zones, k))).pin_memory() for k in names}

    class HZ:
        pass

    hz = HZ()
    for k in names:
        setattr(hz, k, pin[k].numpy())
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.set_zones(hz, stream)
        kn.integrate_batch([g], opts, stream)
        out = g.get(stream)
    e2e_s = time.perf_counter() - t0
    h2d = sum(pin[k].numel() * 8 for k in names)
    d2h = sum(v.nbytes for v in out.values())
    e2e = {"value": steps_per_batch * e2e_steps / e2e_s, "unit": "zone-steps/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "zones_per_s": zones_ok * e2e_steps / e2e_s}

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    kms = _mean(tb["kernel_ms"])
    n_sms = _n_sms()
    if args.form == "fp64":
        roof = fp64_roofline(algorithmic_flops(net, st["steps"], st["rejects"]), kms, kn.measure_fp64_peak(stream),
                             "rates 5 R + fluxes 1/3/7 per 1/2/3-body reaction + gathers S_r + S_p per accepted "
                             "step, 11 N per attempt")
    elif args.form == "qss_fp64":
        roof = fp64_roofline(algorithmic_flops_qss(net, st["steps"], st["rejects"]), kms,
                             kn.measure_fp64_peak(stream),
                             "rates 5 R + fluxes 1/3/7 per 1/2/3-body reaction + gathers S_r + S_p per accepted "
                             "step and again per attempt (the predicted state), 49 N per attempt")
    elif args.form == "mixed_fp64":
        # bound by the FP64 pipe (the update, the conservation sum and the
        # widening of F+ and k); the shared-memory figure rides along
        roof = fp64_roofline(update_fp64_flops(net, st["steps"] + st["rejects"]), kms, kn.measure_fp64_peak(stream),
                             "11 FP64 operations per species per attempt (update, conservation sum, test)")
        roof["smem"] = smem_roofline([(net, st["steps"], st["rejects"])], kms, clk, n_sms)
    else:
        # SM-local bound: shared-memory bandwidth, 32 banks x 4 B per clock per
        # SM at the SM clock sampled during the timed steps
        roof = smem_roofline([(net, st["steps"], st["rejects"])], kms, clk, n_sms, qss=args.form == "qss_mixed")
    # DRAM traffic of the integrator from the committed ncu capture of this
    # kernel (small case, mixed form), scaled to this launch by zone count
    # (each zone's state is read once per launch); null when the kernel's
    # sources changed since the capture, or for another form
    prof = _profile_line("integrate_kernel_mixed_1216x150_full.md")
    traffic = None
    if prof and args.form == "mixed" and prof[2] == kernel_sources_sha256():
        traffic = prof[0] * args.zones / prof[1]
    roof["traffic"] = traffic
    roof["traffic_source"] = ("ncu capture of the mixed-form kernel on 1216 zones (committed summary), "
                              "scaled by zones") if traffic else None
    # the binding resource itself: instruction issue, from the same committed
    # capture (null when the kernel's sources changed since, or another form)
    iss = _profile_issue_line("integrate_kernel_mixed_1216x150_full.md")
    roof["issue"] = None
    if iss and args.form == "mixed" and iss[2] == kernel_sources_sha256():
        roof["issue"] = {"active_frac": iss[0] / 100.0, "lsu_pipe_frac": iss[1] / 100.0,
                         "source": "ncu smsp__issue_active and sm__inst_executed_pipe_lsu of the mixed-form "
                                   "kernel on 1216 zones (committed summary)"}
    if traffic:
        # context: the DRAM side is far from its bound
        peaks, src = _peaks()
        roof["dram_gbs"] = traffic / (kms / 1e3) / 1e9
        roof["dram_frac_of_hbm"] = roof["dram_gbs"] / peaks["hbm_gbs"]
        roof["hbm_peak_source"] = f"MEASURED_PEAKS.json hbm_gbs ({src})"
    groups = None
    if tuned:
        groups = n_sms * (tuned["threads_per_cta"] // tuned["threads_per_zone"])
    elif args.tpz and args.tpc:
        groups = n_sms * (args.tpc // args.tpz)
    dtype = {"mixed": "f32 (float-float state)", "mixed_fp64": "f32 fluxes, f64 update", "fp64": "f64",
             "qss_fp64": "f64", "qss_mixed": "f32 (float-float state)"}[args.form]
    line = {"metric": METRIC, "value": value, "unit": "zone-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if args.strong else "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic", "zones_per_s": zones_all * args.steps / (ms / 1e3),
            "config": {"workload": workload_name(args),
                       "zones_per_gpu": zones.n_zones, "n_species": 150, "n_reactions": 1604,
                       "form": args.form, "l2": "flushed between timed steps (256 MB write)",
                       "accepted_steps_per_batch": int(steps_per_batch), "rejects_per_batch": int(st["rejects"]),
                       "zones_ok": int(zones_ok), "parallelism": f"zones sharded, {world} GPU(s)",
                       "tiling": tuned if tuned else {"threads_per_zone": args.tpz, "threads_per_cta": args.tpc}},
            "clocks": clk, "e2e": e2e, "gpu_launches": 3 * args.steps, "roofline": roof,
            "tail": tail_stats(tb["zone_ns"], zone_steps, groups),
            "paper_context": ("the paper estimates ~100 150-isotope networks integrated on one Kepler GPU "
                              "(Tesla K20X class) in the time an implicit CPU code integrates one (abstract, Sec. 9)")}
    if not args.no_forms and args.form == "mixed":
        line["forms"] = other_forms(kn, g, net, zones, dz, stream, flush,
                                    {"zones_per_s": zones_ok / (kms / 1e3)}, args)
        line["single_zone"] = single_zone_configs()
    if not args.no_cpu:
        exp, be = cpu_baselines(net, zones)
        line["cpu_baseline"] = exp
        line["cpu_implicit_be"] = be
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
