"""Pins of the oracle's accept test, step-size update and step loop (Sec. 4)
against hand-worked cases (tests/golden/accept_test_cases.txt).

The paper gives no error criterion for its adaptive network step; the
library's reading is stated at the top of the golden file.  Each case is
built so that a plausible slip in or_test, or_growth or the loop of
or_integrate changes the outcome: scaling by Y instead of max(Y, Y'), the
y_min cut on one side only or with >=, a signed or per-term-absolute
conservation sum, a dropped mass weight, strict ties, a dropped term of the
growth minimum, shrinking the unclipped step, or growing from it.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from kn_inputs import Zones, custom_network, pair_network

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "accept_test_cases.txt")


def _num(tok):
    if tok in ("nan", "inf", "-inf"):
        return float(tok)
    return float(Fraction(tok))


def _blocks():
    blocks, cur = [], None
    for raw in open(GOLDEN):
        line = raw.strip()
        if not line or line.startswith("#"):
            continue
        head, *rest = line.split()
        if head in ("test", "growth", "trace"):
            cur = {"kind": head, "name": rest[0], "opts": {}}
            blocks.append(cur)
        elif head == "opts":
            cur["opts"] = {k: float(Fraction(v)) for k, v in (kv.split("=") for kv in rest)}
        elif head in ("in", "expect", "zone"):
            cur.setdefault(head, {}).update(dict(kv.split("=") for kv in rest))
        else:
            cur[head] = [_num(x) for x in rest]
    return blocks


def _opts(oracle_mod, kv):
    o = oracle_mod.OracleOpts()
    for k, v in kv.items():
        setattr(o, k, v)
    return o


def _close(got, want, ulps=4):
    if math.isnan(want):
        return math.isnan(got)
    return abs(got - want) <= ulps * 2.0 ** -52 * abs(want)


def test_golden_file_covers_each_part():
    kinds = [b["kind"] for b in _blocks()]
    assert kinds.count("test") >= 10 and kinds.count("growth") >= 5 and kinds.count("trace") >= 1


@pytest.mark.parametrize("case", [b for b in _blocks() if b["kind"] == "test"], ids=lambda b: b["name"])
def test_accept_test_hand_worked(oracle_mod, case):
    A = case["A"]
    net = custom_network(A, [((0,), (0,))], [0.0], [0.0])  # only A is read by the test
    if len(A) > 1:
        net = custom_network(A, [((i,), (i,)) for i in range(len(A))], [0.0] * len(A), [0.0] * len(A))
    orc = oracle_mod.Oracle(net)
    acc, cons, rel, fin = orc.test(case["Y"], case["Yn"], _opts(oracle_mod, case["opts"]))
    e = case["expect"]
    assert acc == bool(int(e["accept"])), case["name"]
    assert fin == bool(int(e["finite"])), case["name"]
    if e["cons"] != "skip":
        assert _close(cons, _num(e["cons"])), (case["name"], cons)
    if e["rel"] != "skip":
        assert _close(rel, _num(e["rel"])), (case["name"], rel)


@pytest.mark.parametrize("case", [b for b in _blocks() if b["kind"] == "growth"], ids=lambda b: b["name"])
def test_growth_hand_worked(oracle_mod, case):
    net = pair_network(1.0, 1.0)
    orc = oracle_mod.Oracle(net)
    g = orc.growth(_num(case["in"]["rel"]), _num(case["in"]["cons"]), _opts(oracle_mod, case["opts"]))
    assert _close(g, _num(case["expect"]["growth"])), (case["name"], g)


@pytest.mark.parametrize("case", [b for b in _blocks() if b["kind"] == "trace"], ids=lambda b: b["name"])
def test_controller_trace_hand_worked(oracle_mod, case):
    net = pair_network(1.0, 1.0)
    assert np.all(net.ln_k0 == 0.0) and np.all(net.t9_exp == 0.0) and np.all(net.A == 1.0)
    zk = {k: _num(v) for k, v in case["zone"].items()}
    z = Zones(Y0=np.array([case["Y0"]]), T0=np.array([1.0]), rho0=np.array([1.0]), tau=np.array([0.0]),
              t_start=np.array([zk["t_start"]]), t_end=np.array([zk["t_end"]]),
              dt_trial=np.array([zk["dt_trial"]]))
    r = oracle_mod.Oracle(net).integrate(z, 0, _opts(oracle_mod, case["opts"]))
    e = case["expect"]
    assert r["steps"] == int(e["steps"]) and r["rejects"] == int(e["rejects"])
    assert r["status"] == int(e["status"])
    assert r["t"] == _num(e["t"])
    assert r["dt_next"] == pytest.approx(_num(e["dt_next"]), rel=1e-13)
    assert np.allclose(r["Y"], case["expect_Y"], rtol=1e-13, atol=0)
