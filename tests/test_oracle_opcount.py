"""The operation count behind the benchmark's roofline (oracle/opcount.py):
the counting scalar's rules on expressions counted by hand, and the stored
table oracle/work_counts.json against a fresh count of the oracle's formulas
(so the work per state the benchmark divides by is reproducible from the
oracle)."""
import json
import math

import numpy as np
import pytest

from oracle import opcount as oc


def _fresh():
    oc._T = oc.Tally()


def _done():
    n = dict(oc._T.n)
    oc._T = None
    return n


def test_counting_rules_on_hand_counted_expressions():
    _fresh()
    x, y, z = oc.Num(2.0), oc.Num(3.0), oc.Num(5.0)
    r = x * y + z                                   # one fused multiply-add
    assert r.v == 11.0
    assert _done() == dict(add=0, mul=0, fma=1, div=0, exp=0, log=0, acc=0)
    _fresh()
    T = oc.Num(1000.0)
    a = 3.0 * T / 2.0 + 7.0                         # constants fold into one fma
    b = np.log(np.array([T], dtype=object))[0]      # ln T
    c = np.log(np.array([T], dtype=object))[0]      # reused
    d = 5.0 / T + 2.0 / (4.0 * T)                   # 1/T once; the sum of two scaled 1/T: a multiply and an fma
    e = T ** 3 + T ** 2                             # T^2 once, T^3 = T^2 T
    f = np.exp(np.array([b * 0.5], dtype=object))[0]
    n = _done()
    assert math.isclose(a.v, 1507.0) and math.isclose(c.v, math.log(1000.0)) and c is b
    assert math.isclose(d.v, 5.0e-3 + 5.0e-4) and math.isclose(e.v, 1.001e9) and math.isclose(f.v, math.sqrt(1000.0))
    assert n["div"] == 1 and n["log"] == 1 and n["exp"] == 1
    assert n["fma"] + n["add"] + n["mul"] == 1 + 2 + 2 + 1 + 1   # a; d's sum; T^2, T^3; e's sum; exp's argument


def test_forward_mode_rules():
    """Derivative columns: a product of values with disjoint columns costs one
    multiply per column; a sum of values sharing a column one add."""
    _fresh()
    x = oc.Num(2.0, frozenset(["x"]))
    y = oc.Num(3.0, frozenset(["y"]))
    p = x * y                                       # value 1, d/dx: *y, d/dy: *x
    n = _done()
    assert p.cols == {"x", "y"} and n["mul"] == 3
    _fresh()
    s = oc.Num(2.0, frozenset(["x"])) + oc.Num(4.0, frozenset(["x"]))
    n = _done()
    assert s.cols == {"x"} and n["add"] == 2        # value + one shared column


@pytest.mark.parametrize("name", ["h2co13", "gri53", "gri53_types", "usc111"])
def test_stored_work_table_is_the_oracle_count(name):
    stored = json.load(open(oc.TABLE))
    assert stored["weights"] == oc.WEIGHTS
    fresh = oc.build_table([name])[name]
    for key, counts in fresh.items():
        if counts is None:
            assert stored["counts"][name][key] is None
            continue
        for cls, v in counts.items():
            assert stored["counts"][name][key][cls] == pytest.approx(v, rel=1e-12), (name, key, cls)


def test_source_count_of_a_one_reaction_mechanism():
    """H + O2 -> OH + O, reversible, elementary, on the 10-species tiny set:
    two exponentials (k_f, and exp(-ln K_c) for k_r), the per-state log of
    T and of P_atm/(R T)... every count is small and the exponentials are
    exactly two."""
    from tests import tiny_mechs as tm
    m = tm.single(dict(reac=[(tm.H, 1), (tm.O2, 1)], prod=[(tm.OH, 1), (tm.O, 1)], A=2.0e11, beta=-0.3,
                       Ea=15000.0))
    c = oc.per_state(m, 0, False, n_states=1)
    assert c["exp"] == 2
    assert c["log"] <= 3
