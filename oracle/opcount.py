"""Operation count of the method, by running the oracle's own formulas on a
counting scalar.

TEST INFRASTRUCTURE ONLY (same rules as ``oracle.kinetics``): imported by the
tests and by ``bench.py``, whose roofline divides the work counted here by a
kernel's time.

``Num`` carries one state's value through ``oracle.kinetics.rates`` and
``source_terms_from_rates`` (numpy object arrays of ``Num``) and tallies the
FP64 operations an evaluation of those formulas needs, per class:

* add (also subtract), mul, fma (a product consumed by an addition is fused,
  as compilers contract them), div, exp, log;
* arithmetic on mechanism constants alone is free (done once per mechanism);
  a product with a constant is carried as a pending scale and folds into the
  fused multiply-add or the next product that consumes it; multiplying by
  +-1 and adding 0 are free;
* per state, ln x, 1/x and integer powers x^n of one value are formed once
  and reused (ln T, 1/T, T^2 .. T^4 of the thermodynamic polynomials);
  x^c for non-integer c is exp(c ln x), 10^x is exp(x ln 10), log10 is a
  log and a multiply.

With ``derivatives=True`` every ``Num`` also carries the set of state
variables it depends on, and each operation adds the forward-mode
chain-rule work for the derivative columns it produces (Sec. 2.2's
Jacobian J_ij = df_i/dPhi_j, column by column): for a sum one add per
column both operands carry; for a product one multiply per column of one
operand and a multiply plus a fused multiply-add per shared column; for a
quotient the same with the reciprocal; for exp, log and powers one multiply
per column (after forming the local derivative).  The additions that merge
per-reaction derivative contributions into a running sum are tallied apart
("acc"): they are the Jacobian entry accumulations.
"""
from __future__ import annotations

import math

import numpy as np

CLASSES = ("add", "mul", "fma", "div", "exp", "log", "acc")


class Tally:
    def __init__(self):
        self.n = dict.fromkeys(CLASSES, 0)
        self.memo = {}

    def add(self, cls, k=1):
        self.n[cls] += k


_T: Tally | None = None


def _is_num(x):
    return isinstance(x, Num)


class Num:
    """One FP64 value of a state's evaluation (see the module notes)."""
    __slots__ = ("v", "cols", "lazy", "prod", "sumlike", "base")

    def __init__(self, v, cols=frozenset(), lazy=False, prod=False, sumlike=False, base=None):
        self.v = float(v)
        self.cols = cols          # state variables this value depends on
        self.lazy = lazy          # carries a pending constant factor (one multiply owed)
        self.prod = prod          # an unconsumed product of two state values (fusable)
        self.sumlike = sumlike    # a running sum of contributions
        # the value without its pending constant factor (lazy values): the
        # key of reciprocals and logarithms, so that 1/(c x) and ln(c x)
        # reuse 1/x and ln x
        self.base = self.v if base is None else float(base)

    # -- helpers -------------------------------------------------------------
    def _materialise(self):
        if self.lazy:
            _T.add("mul")
            _T.add("mul", len(self.cols))
            return Num(self.v, self.cols)
        return self

    def _consume_product(self):
        """A product consumed by an addition: its multiply becomes an fma."""
        if self.prod:
            self.prod = False
            return True
        return False

    # -- arithmetic -----------------------------------------------------------
    def __add__(self, o):
        if not _is_num(o):
            if o == 0:
                # a sum that starts from zero: a running accumulation
                return Num(self.v, self.cols, self.lazy, self.prod, sumlike=True)
            # constant + value: one add (an fma when the value owes a scale)
            if self.lazy:
                _T.add("fma")
                return Num(self.v + o, self.cols)
            if self._consume_product():
                _T.add("fma")
                _T.n["mul"] -= 1
            else:
                _T.add("add")
            return Num(self.v + o, self.cols)
        a, b = self, o
        fused = 0
        for x in (a, b):
            if x.lazy:
                fused += 1
        if fused == 2:
            _T.add("mul")
            fused = 1
        if fused == 0:
            if a._consume_product() or b._consume_product():
                _T.n["mul"] -= 1
                fused = 1
        _T.add("fma" if fused else "add")
        shared = a.cols & b.cols
        # derivative columns: one add per column both carry
        if a.sumlike or b.sumlike:
            _T.add("acc", len(shared))
        else:
            _T.add("add", len(shared))
        # a lazily scaled operand's own columns need the scale
        for x in (a, b):
            if x.lazy:
                _T.add("mul", len(x.cols - shared))
        return Num(a.v + b.v, a.cols | b.cols, sumlike=a.sumlike or b.sumlike)

    __radd__ = __add__

    def __neg__(self):
        return Num(-self.v, self.cols, self.lazy, self.prod, self.sumlike, self.base)

    def __sub__(self, o):
        return self + (-o)

    def __rsub__(self, o):
        return (-self) + o

    def __mul__(self, o):
        if not _is_num(o):
            if o == 0:
                return 0.0
            if o == 1:
                return self
            if o == -1:
                return -self
            return Num(self.v * o, self.cols, lazy=True, base=self.base)
        a, b = self, o
        # a pending constant factor commutes into the product
        lazy = a.lazy or b.lazy
        if a.lazy and b.lazy:
            pass  # both scales are constants: their product is a constant
        _T.add("mul")
        shared = a.cols & b.cols
        _T.add("mul", len((a.cols | b.cols) - shared))
        _T.add("mul", len(shared))
        _T.add("fma", len(shared))
        return Num(a.v * b.v, a.cols | b.cols, lazy=lazy, prod=not lazy, base=a.base * b.base)

    __rmul__ = __mul__

    def recip(self):
        """1/self, formed once per value (1/(c x) = (1/c) (1/x) reuses 1/x)."""
        key = ("recip", self.base, self.cols)
        hit = _T.memo.get(key)
        if hit is None:
            _T.add("div")
            if self.cols:
                _T.add("mul")                   # -1/x^2
                _T.add("mul", len(self.cols))
            hit = Num(1.0 / self.base, self.cols)
            _T.memo[key] = hit
        if self.lazy:
            return Num(1.0 / self.v, self.cols, lazy=True, base=hit.v)
        return hit

    def __truediv__(self, o):
        if not _is_num(o):
            return self * (1.0 / o)
        return self * o.recip()

    def __rtruediv__(self, o):
        r = self.recip()
        return r * o

    def __pow__(self, e):
        if _is_num(e):
            return (e * self.log()).exp()
        if float(e).is_integer():
            k = int(e)
            if k == 0:
                return 1.0
            if k == 1:
                return self
            if k < 0:
                return self.recip() ** (-k)
            key = ("pow", self.base, self.cols, k)
            hit = _T.memo.get(key)
            if hit is None:
                base = Num(self.base, self.cols)
                prev = base if k == 2 else base ** (k - 1)
                hit = prev * base
                hit.prod = False
                _T.memo[key] = hit
            if self.lazy:
                return Num(self.v ** k, self.cols, lazy=True, base=hit.v)
            return hit
        return (e * self.log()).exp()

    def __rpow__(self, b):
        return (self * math.log(b)).exp()

    def exp(self):
        x = self._materialise()
        _T.add("exp")
        _T.add("mul", len(x.cols))
        return Num(math.exp(x.v) if x.v < 709 else float("inf"), x.cols)

    def log(self):
        """ln self, formed once per value (ln(c x) = ln c + ln x reuses ln x)."""
        key = ("log", self.base, self.cols)
        hit = _T.memo.get(key)
        if hit is None:
            _T.add("log")
            if self.cols:
                Num(self.base, self.cols).recip()   # d ln x = dx / x
                _T.add("mul", len(self.cols))
            hit = Num(math.log(self.base), self.cols)
            _T.memo[key] = hit
        if self.lazy:
            _T.add("add")                            # + ln c
            return Num(math.log(self.v), self.cols)
        return hit

    def log10(self):
        return self.log() * (1.0 / math.log(10.0))

    # -- comparisons and conversions (free) ----------------------------------
    def __lt__(self, o):
        return self.v < (o.v if _is_num(o) else o)

    def __le__(self, o):
        return self.v <= (o.v if _is_num(o) else o)

    def __gt__(self, o):
        return self.v > (o.v if _is_num(o) else o)

    def __ge__(self, o):
        return self.v >= (o.v if _is_num(o) else o)

    def __abs__(self):
        return Num(abs(self.v), self.cols, self.lazy, self.prod, self.sumlike)

    def __float__(self):
        return self.v

    def __bool__(self):
        return self.v != 0.0


class Seed(Num):
    """A zero that only attaches a derivative column: adding it is free."""
    __slots__ = ()

    def __add__(self, o):
        if _is_num(o):
            return Num(o.v, o.cols | self.cols, o.lazy, o.prod, o.sumlike, o.base)
        return Num(o, self.cols)

    __radd__ = __add__


def count(mech, mode, phi, param, derivatives=False):
    """Operation counts (dict over CLASSES) of one state's source terms
    (derivatives=True: source terms and Jacobian, forward mode), state given
    as phi [N] and param (P in CONP, V in CONV).

    The derivatives are taken with respect to the rates' own variables: T,
    the state variable S (V or P), and each concentration C_k with the bath
    gas's C_Ns as one more column.  The Jacobian's species columns follow
    from these by dq/dn_j = (dq/dC_j - dq/dC_Ns) / V (Sec. 2.2: C_Ns =
    C_tot - sum C_k), one subtraction per entry, which the accumulation of
    the entries carries ("acc")."""
    from . import kinetics as K
    global _T
    _T = Tally()
    try:
        N = phi.shape[0]
        ns = mech.n_species
        x = np.empty((N, 1), dtype=object)
        for j in range(N):
            cols = frozenset([("x", j)]) if derivatives and j < 2 else frozenset()
            x[j, 0] = Num(phi[j], cols)
        p = np.empty(1, dtype=object)
        p[0] = Num(param)              # a per-state input, not differentiated
        dC = None
        if derivatives:
            dC = np.empty((ns, 1), dtype=object)
            for k in range(ns):
                dC[k, 0] = Seed(0.0, frozenset([("C", k)]))
        r = K.rates(mech, mode, x, p, dC=dC)
        f, _ = K.source_terms_from_rates(mech, mode, r)
        for v in f.ravel():
            if _is_num(v):
                v._materialise()
        if derivatives:
            # species columns from the concentration columns: one entry
            # update per structural nonzero of the species block
            nz = int(K.sparsity_pattern(mech)[2:, 2:].sum())
            _T.add("acc", nz)
        return dict(_T.n)
    finally:
        _T = None


# FP64 cost of one operation of each class in DFMA issue slots: add, multiply
# and fused multiply-add 1; the kernels' table-driven exp 9 (reduction 3,
# polynomial 4, table product 1, exponent shift 1); CUDA's log 30.2 and
# divide 5.7, measured on this GB300.
WEIGHTS = dict(add=1.0, mul=1.0, fma=1.0, div=5.7, exp=9.0, log=30.2, acc=1.0)


def work(counts, weights=WEIGHTS, with_acc=False):
    """DFMA-equivalent FP64 work of a count (accumulations excluded unless
    with_acc: the kernels do them as L2 reductions, off the FP64 pipe)."""
    return sum(weights[c] * counts[c] for c in CLASSES if c != "acc" or with_acc)


def per_state(mech, mode=0, derivatives=False, n_states=4, seed=7):
    """Mean counts over a few states of the workload recipe (the NASA-7 range
    and nothing else depends on the state)."""
    import synth
    phi, par = synth.make_states(mech, n_states, seed, mode)
    tot = dict.fromkeys(CLASSES, 0.0)
    for s in range(n_states):
        c = count(mech, mode, phi[:, s], par[s], derivatives)
        for k in CLASSES:
            tot[k] += c[k] / n_states
    return tot


# ---------------------------------------------------------------------------
# the table bench.py divides by (oracle/work_counts.json), written by
#   python -m oracle.opcount
# ---------------------------------------------------------------------------
TABLE = __import__("os").path.join(__import__("os").path.dirname(__file__), "work_counts.json")
TABLE_MECHS = ("h2co13", "gri53", "gri53_types", "usc111", "ic5874")


def lu_counts(mech):
    """Operations of one factorisation of the Newton matrix in the fixed fill
    pattern of oracle.linalg.lu_symbolic: per pivot k one reciprocal of the
    pivot, a multiply per entry below it (the column scaling) and a fused
    multiply-add per (row below, column right) pair of the fill pattern."""
    from .linalg import lu_symbolic
    _, F, _ = lu_symbolic(mech)
    N = F.shape[0]
    fma = mul = 0
    for k in range(N):
        rows = int(F[k + 1:, k].sum())
        cols = int(F[k, k + 1:].sum())
        mul += rows
        fma += rows * cols
    return dict(add=0, mul=mul, fma=fma, div=N, exp=0, log=0, acc=0)


def newton_lu_counts(mech):
    """The LU of M = I - h gamma J formed from the Jacobian's values
    (oracle.forms.newton_matrix, evaluated over the Jacobian's pattern): one
    multiply per stored Jacobian entry and one add per diagonal entry, then
    the factorisation of lu_counts."""
    from .kinetics import sparsity_pattern
    c = dict(lu_counts(mech))
    c["mul"] += int(sparsity_pattern(mech).sum())
    c["add"] += mech.n_species + 1
    return c


def build_table(names=TABLE_MECHS):
    """{mechanism: {"source": counts, "jacobian": counts, "lu": counts,
    "newton_lu": counts}},
    counts per state (mean of the states of per_state) in CONP and CONV."""
    import synth
    out = {}
    for name in names:
        m = synth.make_mechanism(name)
        e = {}
        for mode, tag in ((0, "conp"), (1, "conv")):
            n_states = 2 if m.n_species < 200 else 1
            e[f"source_{tag}"] = per_state(m, mode, False, n_states=n_states)
            e[f"jacobian_{tag}"] = per_state(m, mode, True, n_states=n_states)
        e["lu"] = lu_counts(m) if m.n_species < 200 else None
        e["newton_lu"] = newton_lu_counts(m) if m.n_species < 200 else None
        out[name] = e
    return out


def load_table():
    import json
    with open(TABLE) as f:
        return json.load(f)


if __name__ == "__main__":
    import json
    import sys
    names = sys.argv[1:] or TABLE_MECHS
    table = build_table(names)
    with open(TABLE, "w") as f:
        json.dump({"weights": WEIGHTS, "counts": table}, f, indent=1, sort_keys=True)
    print(f"wrote {TABLE}")
