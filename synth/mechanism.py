"""Seeded synthetic chemical mechanisms.

The paper measures on four real mechanisms (H2/CO, GRI-Mech 3.0, USC-Mech II,
iC5H11OH; Sec. 3.1, Table "t:models") and partially-stirred-reactor state
databases.  None of those are available, so this module builds random
mechanisms of the same sizes from a stated recipe:

* species: element compositions over H, O, C, N, Ar drawn from a small-molecule
  lattice, with N2 as the last species (the bath gas of the state vector,
  Sec. 2.2);
* NASA 7-coefficient polynomials in two temperature ranges, least-squares fits
  of a smooth Einstein-oscillator heat capacity, with the enthalpy and entropy
  constants set from a random formation enthalpy / entropy and made continuous
  at T_mid;
* element-balanced reactions with one or two reactants and one or two products,
  written in the exothermic direction, with modified-Arrhenius parameters
  ln A ~ U[10, 40], beta ~ U[-2, 3], Ea ~ U[0, 50000] cal/mol, a reversible
  fraction, and third-body / Lindemann / Troe / SRI pressure dependence.

This module is an input generator shared by the oracle and by the CUDA path.
It holds none of the evaluated method's arithmetic: it writes mechanism data,
it never evaluates rates, source terms or Jacobians.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

ELEMENTS = ("H", "O", "C", "N", "AR")
# IUPAC conventional atomic weights, kg/kmol
ATOMIC_MASS = np.array([1.008, 15.999, 12.011, 14.007, 39.948])
R_GAS = 8314.46261815324  # J / (kmol K)

# reaction kinds
ELEMENTARY, THIRD_BODY, LINDEMANN, TROE, SRI, PLOG, CHEB = 0, 1, 2, 3, 4, 5, 6
KIND_NAMES = {ELEMENTARY: "ELEMENTARY", THIRD_BODY: "THIRD_BODY", LINDEMANN: "LINDEMANN", TROE: "TROE",
              SRI: "SRI", PLOG: "PLOG", CHEB: "CHEBYSHEV"}
MAX_SP = 4  # distinct species per reaction side supported by the format


@dataclass
class Mechanism:
    """Plain mechanism data (0-based indices; species Ns-1 is the bath gas).

    Units: W kg/kmol; NASA-7 coefficients dimensionless (cp/R form, T in K);
    A in (m^3/kmol)^(order-1)/s with order the reactant molecularity (+1 for a
    third body or for the low-pressure limit of a falloff reaction); Ea in
    cal/mol.
    """
    name: str
    species: list
    composition: np.ndarray          # int [Ns, Ne]
    W: np.ndarray                    # [Ns]
    T_mid: np.ndarray                # [Ns]
    nasa_low: np.ndarray             # [Ns, 7]
    nasa_high: np.ndarray            # [Ns, 7]
    kind: np.ndarray                 # int [Nr]
    reversible: np.ndarray           # bool [Nr]
    reac_sp: np.ndarray              # int [Nr, MAX_SP], -1 padded
    reac_nu: np.ndarray              # int [Nr, MAX_SP]
    prod_sp: np.ndarray              # int [Nr, MAX_SP]
    prod_nu: np.ndarray              # int [Nr, MAX_SP]
    A: np.ndarray                    # [Nr] (high-pressure limit for falloff)
    beta: np.ndarray
    Ea: np.ndarray
    A0: np.ndarray                   # [Nr] low-pressure limit (falloff only)
    beta0: np.ndarray
    Ea0: np.ndarray
    troe: np.ndarray                 # [Nr, 4]: a, T3, T1, T2
    troe_n: np.ndarray               # int [Nr]: 3 or 4 Troe parameters
    sri: np.ndarray                  # [Nr, 5]: a, b, c, d, e
    eff_ptr: np.ndarray              # int [Nr+1] CSR of non-default efficiencies
    eff_sp: np.ndarray               # int [n_eff]
    eff_val: np.ndarray              # [n_eff] absolute efficiency alpha
    elements: tuple = ELEMENTS
    # less common reaction types (absent unless given)
    chem: np.ndarray = None          # bool [Nr]: chemically-activated falloff (rate k0 F / (1 + Pr))
    rev_explicit: np.ndarray = None  # bool [Nr]: reverse rate from rev_arr instead of K_c
    rev_arr: np.ndarray = None       # [Nr, 3]: reverse A, beta, Ea
    plog_ptr: np.ndarray = None      # int [Nr+1]: P-log entries of each reaction
    plog: np.ndarray = None          # [n_plog, 4]: P [Pa], A, beta, Ea; P ascending per reaction
    cheb_ptr: np.ndarray = None      # int [Nr+1]: offsets into cheb_coef
    cheb_shape: np.ndarray = None    # int [Nr, 2]: N_T, N_P
    cheb_range: np.ndarray = None    # [Nr, 4]: T_min, T_max [K], P_min, P_max [Pa]
    cheb_coef: np.ndarray = None     # row-major N_T x N_P per reaction: log10 k, k in SI-kmol units

    def __post_init__(self):
        nr = len(self.kind)
        if self.chem is None:
            self.chem = np.zeros(nr, dtype=bool)
        if self.rev_explicit is None:
            self.rev_explicit = np.zeros(nr, dtype=bool)
        if self.rev_arr is None:
            self.rev_arr = np.zeros((nr, 3))
        if self.plog_ptr is None:
            self.plog_ptr = np.zeros(nr + 1, dtype=np.int64)
        if self.plog is None:
            self.plog = np.zeros((0, 4))
        if self.cheb_ptr is None:
            self.cheb_ptr = np.zeros(nr + 1, dtype=np.int64)
        if self.cheb_shape is None:
            self.cheb_shape = np.zeros((nr, 2), dtype=np.int64)
        if self.cheb_range is None:
            self.cheb_range = np.zeros((nr, 4))
        if self.cheb_coef is None:
            self.cheb_coef = np.zeros(0)

    def plog_table(self, i: int) -> np.ndarray:
        return self.plog[self.plog_ptr[i]:self.plog_ptr[i + 1]]

    def cheb_table(self, i: int) -> np.ndarray:
        nT, nP = self.cheb_shape[i]
        return self.cheb_coef[self.cheb_ptr[i]:self.cheb_ptr[i + 1]].reshape(nT, nP)

    @property
    def n_species(self) -> int:
        return len(self.species)

    @property
    def n_reactions(self) -> int:
        return len(self.kind)

    def efficiencies(self, i: int) -> dict:
        lo, hi = self.eff_ptr[i], self.eff_ptr[i + 1]
        return {int(k): float(v) for k, v in zip(self.eff_sp[lo:hi], self.eff_val[lo:hi])}

    def reactants(self, i: int) -> list:
        return [(int(k), int(n)) for k, n in zip(self.reac_sp[i], self.reac_nu[i]) if k >= 0]

    def products(self, i: int) -> list:
        return [(int(k), int(n)) for k, n in zip(self.prod_sp[i], self.prod_nu[i]) if k >= 0]

    def copy(self) -> "Mechanism":
        return dataclasses.replace(self, **{f.name: (getattr(self, f.name).copy()
                                    if isinstance(getattr(self, f.name), np.ndarray)
                                    else getattr(self, f.name))
                                    for f in dataclasses.fields(self)})


# --------------------------------------------------------------------------
# workload recipes (sizes and reaction-kind fractions of the measured cases)
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class MechSpec:
    name: str
    n_species: int
    n_reactions: int
    f_third_body: float
    f_troe: float
    f_lindemann: float
    f_sri: float
    seed: int
    f_reversible: float = 0.9
    # less common reaction types, converted from the plain mechanism of the
    # same seed: P-log and Chebyshev replace elementary reactions,
    # chemically-activated falloff a fraction of the falloff reactions,
    # explicit reverse Arrhenius parameters a fraction of the reversible ones
    f_plog: float = 0.0
    f_cheb: float = 0.0
    f_chem: float = 0.0
    f_rev_explicit: float = 0.0


SPECS = {
    "h2co13": MechSpec("h2co13", 13, 27, 0.15, 0.10, 0.0, 0.0, seed=1809 + 1),
    "gri53": MechSpec("gri53", 53, 325, 0.10, 0.08, 0.02, 0.01, seed=1809 + 2),
    "usc111": MechSpec("usc111", 111, 784, 0.10, 0.08, 0.02, 0.01, seed=1809 + 3),
    "ic5874": MechSpec("ic5874", 874, 3796, 0.12, 0.10, 0.02, 0.01, seed=1809 + 5),
    # the 53/325 mechanism with every less common type (none of the paper's
    # workloads has them): 5 % P-log, 3 % Chebyshev, a third of the falloff
    # reactions chemically activated, 10 % of the reversible reactions with
    # explicit reverse parameters
    "gri53_types": MechSpec("gri53_types", 53, 325, 0.10, 0.08, 0.02, 0.01, seed=1809 + 2,
                            f_plog=0.05, f_cheb=0.03, f_chem=1.0 / 3.0, f_rev_explicit=0.10),
}


def _formula(c) -> str:
    s = ""
    for e, n in zip(ELEMENTS, c):
        if n:
            s += e + (str(int(n)) if n > 1 else "")
    return s


def _species_compositions(rng, ns: int) -> np.ndarray:
    """ns distinct compositions; the last one is N2 (bath gas)."""
    bath = (0, 0, 0, 2, 0)
    if ns <= 16:
        lim = (3, 2, 1, 2)
    elif ns <= 64:
        lim = (4, 3, 2, 2)
    elif ns <= 128:
        lim = (6, 3, 3, 2)
    else:
        lim = (14, 4, 9, 2)
    pts = []
    for h in range(lim[0] + 1):
        for o in range(lim[1] + 1):
            for c in range(lim[2] + 1):
                for n in range(lim[3] + 1):
                    t = (h, o, c, n, 0)
                    if sum(t) == 0 or t == bath:
                        continue
                    pts.append(t)
    pts.append((0, 0, 0, 0, 1))  # argon
    pts = np.array(pts)
    natoms = pts.sum(1)
    w = np.exp(-0.25 * natoms) * np.where(pts[:, 3] > 0, 0.1, 1.0)
    # atoms and diatomics first make balanced reactions plentiful
    must = [i for i, p in enumerate(pts) if tuple(p) in
            {(1, 0, 0, 0, 0), (0, 1, 0, 0, 0), (2, 0, 0, 0, 0), (0, 2, 0, 0, 0),
             (1, 1, 0, 0, 0), (2, 1, 0, 0, 0)}]
    rest = [i for i in range(len(pts)) if i not in must]
    pr = w[rest] / w[rest].sum()
    pick = list(rng.choice(rest, size=ns - 1 - len(must), replace=False, p=pr))
    comp = np.vstack([pts[must], pts[pick], np.array(bath)[None, :]])
    return comp.astype(np.int64)


def _einstein_cp(T, c0, c1, theta):
    x = theta / T
    ex = np.exp(x)
    return c0 + c1 * x * x * ex / (ex - 1.0) ** 2


def _fit_nasa(rng, comp, T_low=300.0, T_mid=1000.0, T_high=3500.0,
              bath=False):
    """NASA-7 coefficient pairs fit to a smooth cp(T), continuous at T_mid."""
    na = int(comp.sum())
    if na == 1:
        c0, c1 = 2.5, rng.uniform(0.0, 0.2)
    elif na == 2:
        c0, c1 = 3.5, rng.uniform(0.7, 1.0)
    else:
        c0, c1 = 4.0, (3 * na - 6) * rng.uniform(0.6, 0.95)
    theta = rng.uniform(600.0, 2500.0)
    coef = []
    for lo, hi in ((T_low, T_mid), (T_mid, T_high)):
        T = np.linspace(lo, hi, 200)
        wts = np.ones_like(T)
        wts[np.argmin(np.abs(T - T_mid))] = 1e3
        x = T / 1000.0
        V = np.vander(x, 5, increasing=True) * wts[:, None]
        b, *_ = np.linalg.lstsq(V, _einstein_cp(T, c0, c1, theta) * wts, rcond=None)
        coef.append(b / 1000.0 ** np.arange(5))
    a_lo, a_hi = coef
    # enthalpy / entropy integration constants (NASA-7 definition)
    if bath:
        hf_R, s_R = 0.0, 191.6e3 / R_GAS
    else:
        hf_R = rng.uniform(-120e6, 220e6) / R_GAS
        s_R = rng.uniform(13.0, 20.0) + 2.2 * min(na, 12)

    def hpoly(a, T):  # integral of cp/R dT without the constant
        return a[0] * T + a[1] * T ** 2 / 2 + a[2] * T ** 3 / 3 + a[3] * T ** 4 / 4 + a[4] * T ** 5 / 5

    def spoly(a, T):  # integral of cp/(R T) dT without the constant
        return a[0] * np.log(T) + a[1] * T + a[2] * T ** 2 / 2 + a[3] * T ** 3 / 3 + a[4] * T ** 4 / 4

    a5_lo = hf_R - hpoly(a_lo, 298.15)
    a6_lo = s_R - spoly(a_lo, 298.15)
    a5_hi = hpoly(a_lo, T_mid) + a5_lo - hpoly(a_hi, T_mid)
    a6_hi = spoly(a_lo, T_mid) + a6_lo - spoly(a_hi, T_mid)
    low = np.concatenate([a_lo, [a5_lo, a6_lo]])
    high = np.concatenate([a_hi, [a5_hi, a6_hi]])
    return low, high, hf_R


def _balanced_reactions(rng, comp, nr, hf, n_hub=6, p_hub=0.9):
    """nr distinct element-balanced reactions (1-2 reactants, 1-2 products).

    Like real mechanisms, most reactions involve one of the small "hub"
    species (the first n_hub: H, O, H2, O2, OH, H2O) on each side: with
    probability p_hub a candidate without a hub on both sides is rejected.
    """
    ns = len(comp)
    groups = {}
    for a in range(ns):
        groups.setdefault(comp[a].tobytes(), []).append((a,))
    for a in range(ns):
        ca = comp[a]
        for b in range(a, ns):
            groups.setdefault((ca + comp[b]).tobytes(), []).append((a, b))
    multi = [g for g in groups.values() if len(g) >= 2]
    if not multi:
        return None
    sizes = np.array([len(g) * (len(g) - 1) / 2 for g in multi], dtype=float)
    p = sizes / sizes.sum()
    chosen, seen = [], set()
    tries = 0
    while len(chosen) < nr and tries < 200 * nr + 10000:
        tries += 1
        g = multi[rng.choice(len(multi), p=p)]
        i, j = rng.choice(len(g), size=2, replace=False)
        r, q = g[i], g[j]
        if set(r) & set(q):
            continue
        key = tuple(sorted((r, q)))
        if key in seen:
            continue
        hub_r = any(k < n_hub for k in r)
        hub_q = any(k < n_hub for k in q)
        if not (hub_r and hub_q) and rng.random() < p_hub:
            continue
        seen.add(key)
        # exothermic direction (formation-enthalpy difference at 298 K)
        dh = sum(hf[k] for k in q) - sum(hf[k] for k in r)
        if dh > 0:
            r, q = q, r
        chosen.append((r, q))
    if len(chosen) < nr:
        return None
    return chosen


def make_mechanism(spec: MechSpec | str) -> Mechanism:
    """Build the seeded synthetic mechanism of a recipe (deterministic)."""
    if isinstance(spec, str):
        spec = SPECS[spec]
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    ns, nr = spec.n_species, spec.n_reactions
    for _attempt in range(50):
        comp = _species_compositions(rng, ns)
        low = np.zeros((ns, 7))
        high = np.zeros((ns, 7))
        hf = np.zeros(ns)
        for k in range(ns):
            low[k], high[k], hf[k] = _fit_nasa(rng, comp[k], bath=(k == ns - 1))
        rx = _balanced_reactions(rng, comp, nr, hf)
        if rx is not None:
            break
    else:
        raise RuntimeError(f"could not build {nr} balanced reactions for {ns} species")
    W = comp @ ATOMIC_MASS
    names = [_formula(c) for c in comp]

    kind = np.full(nr, ELEMENTARY, dtype=np.int64)
    # pressure dependence goes preferentially to association/dissociation
    assoc = [i for i, (r, q) in enumerate(rx) if len(r) != len(q)]
    other = [i for i in range(nr) if i not in set(assoc)]
    order = list(rng.permutation(assoc)) + list(rng.permutation(other))
    counts = [(TROE, spec.f_troe), (LINDEMANN, spec.f_lindemann),
              (SRI, spec.f_sri), (THIRD_BODY, spec.f_third_body)]
    pos = 0
    for kd, f in counts:
        c = int(round(f * nr))
        for i in order[pos:pos + c]:
            kind[i] = kd
        pos += c

    reversible = rng.random(nr) < spec.f_reversible
    reac_sp = np.full((nr, MAX_SP), -1, dtype=np.int64)
    reac_nu = np.zeros((nr, MAX_SP), dtype=np.int64)
    prod_sp = np.full((nr, MAX_SP), -1, dtype=np.int64)
    prod_nu = np.zeros((nr, MAX_SP), dtype=np.int64)
    for i, (r, q) in enumerate(rx):
        for side_sp, side_nu, ms in ((reac_sp, reac_nu, r), (prod_sp, prod_nu, q)):
            uniq = sorted(set(ms))
            for s, k in enumerate(uniq):
                side_sp[i, s] = k
                side_nu[i, s] = ms.count(k)

    lnA = rng.uniform(10.0, 40.0, nr)
    beta = rng.uniform(-2.0, 3.0, nr)
    Ea = rng.uniform(0.0, 50000.0, nr)
    fall = np.isin(kind, (LINDEMANN, TROE, SRI))
    lnA0 = np.where(fall, lnA + rng.uniform(2.0, 12.0, nr), 0.0)
    beta0 = np.where(fall, beta - rng.uniform(0.0, 2.0, nr), 0.0)
    Ea0 = np.where(fall, Ea * rng.uniform(0.0, 0.8, nr), 0.0)
    A0 = np.where(fall, np.exp(lnA0), 0.0)

    troe = np.zeros((nr, 4))
    troe_n = np.zeros(nr, dtype=np.int64)
    sri = np.zeros((nr, 5))
    for i in range(nr):
        if kind[i] == TROE:
            has_t2 = rng.random() < 0.5
            troe[i] = (rng.uniform(0.05, 0.95), np.exp(rng.uniform(np.log(30), np.log(1000))),
                       np.exp(rng.uniform(np.log(300), np.log(1e4))),
                       np.exp(rng.uniform(np.log(500), np.log(1e4))) if has_t2 else 0.0)
            troe_n[i] = 4 if has_t2 else 3
        elif kind[i] == SRI:
            sri[i] = (rng.uniform(0.2, 2.0), rng.uniform(50.0, 800.0), rng.uniform(100.0, 3000.0),
                      rng.uniform(0.5, 1.5) if rng.random() < 0.5 else 1.0,
                      rng.uniform(-0.5, 0.5) if rng.random() < 0.5 else 0.0)

    # a shared set of colliders with non-default third-body efficiencies, as
    # in real mechanisms (H2, H2O, CO, ... carry the same efficiencies in
    # every pressure-dependent reaction); each reaction picks up to 3 of them
    colliders = rng.choice(ns - 1, size=min(6, ns - 1), replace=False)
    # a non-unit bath-gas efficiency makes whole Jacobian rows dense (Sec. 3.4);
    # it is kept to about four reactions per mechanism (probability <= 0.1)
    n_pd = int(np.sum(kind != ELEMENTARY))
    p_bath = min(0.1, 4.0 / max(n_pd, 1))
    eff_ptr = [0]
    eff_sp, eff_val = [], []
    for i in range(nr):
        if kind[i] != ELEMENTARY:
            picks = set(rng.choice(colliders, size=min(3, len(colliders)), replace=False).tolist())
            if rng.random() < p_bath:
                picks.add(ns - 1)
            for k in sorted(picks):
                eff_sp.append(k)
                eff_val.append(rng.uniform(0.0, 5.0))
        eff_ptr.append(len(eff_sp))

    m = Mechanism(
        name=spec.name, species=names, composition=comp, W=W,
        T_mid=np.full(ns, 1000.0), nasa_low=low, nasa_high=high,
        kind=kind, reversible=reversible,
        reac_sp=reac_sp, reac_nu=reac_nu, prod_sp=prod_sp, prod_nu=prod_nu,
        A=np.exp(lnA), beta=beta, Ea=Ea, A0=A0, beta0=beta0, Ea0=Ea0,
        troe=troe, troe_n=troe_n, sri=sri,
        eff_ptr=np.array(eff_ptr, dtype=np.int64), eff_sp=np.array(eff_sp, dtype=np.int64),
        eff_val=np.array(eff_val, dtype=float))
    if spec.f_plog or spec.f_cheb or spec.f_chem or spec.f_rev_explicit:
        _add_special_types(m, spec)
    return m


P_ATM = 101325.0


def _add_special_types(m: Mechanism, spec: MechSpec) -> None:
    """Convert reactions of a plain mechanism to the less common types (a
    separate random stream, so the plain reactions stay those of the plain
    recipe with the same seed).

    * P-log: 2-5 pressures log-spaced over [0.01, 100] atm; entry m has
      ln A_m = ln A + U[-2, 2] + g (m - centre) with g ~ U[-0.5, 0.5], beta_m
      = beta + U[-0.3, 0.3], Ea_m = Ea U[0.9, 1.1].
    * Chebyshev: N_T x N_P in {4..7} x {2..4}, T in [300, 3000] K, P in
      [0.01, 100] atm; a_00 ~ U[8, 12] (log10 k), a_10 ~ U[-1.5, -0.2], the
      other coefficients N(0, 0.3 / (1 + t + p)^2).
    * chemically activated: the falloff parameters unchanged, the rate
      becomes k0 F / (1 + Pr).
    * explicit reverse: ln A_r = ln A + U[-3, 3], beta_r = beta + U[-0.5, 0.5],
      Ea_r = Ea + U[0, 30000] cal/mol.
    """
    rng = np.random.Generator(np.random.PCG64(spec.seed + 7000))
    nr = m.n_reactions
    elem = [i for i in range(nr) if m.kind[i] == ELEMENTARY]
    n_plog = int(round(spec.f_plog * nr))
    n_cheb = int(round(spec.f_cheb * nr))
    pick = rng.permutation(elem)[:n_plog + n_cheb]
    plog_set = set(int(i) for i in pick[:n_plog])
    cheb_set = set(int(i) for i in pick[n_plog:])
    plog, cheb = [], []
    for i in range(nr):
        if i in plog_set:
            m.kind[i] = PLOG
            npts = int(rng.integers(2, 6))
            Ps = P_ATM * np.logspace(-2.0, 2.0, npts)
            g = rng.uniform(-0.5, 0.5)
            lnA = np.log(m.A[i])
            for j, P in enumerate(Ps):
                plog.append([P, np.exp(lnA + rng.uniform(-2.0, 2.0) + g * (j - (npts - 1) / 2)),
                             m.beta[i] + rng.uniform(-0.3, 0.3), m.Ea[i] * rng.uniform(0.9, 1.1)])
        m.plog_ptr[i + 1] = len(plog)
        if i in cheb_set:
            m.kind[i] = CHEB
            nT, nP = int(rng.integers(4, 8)), int(rng.integers(2, 5))
            t, q = np.meshgrid(np.arange(nT), np.arange(nP), indexing="ij")
            a = rng.standard_normal((nT, nP)) * 0.3 / (1.0 + t + q) ** 2
            a[0, 0] = rng.uniform(8.0, 12.0)
            a[1, 0] = rng.uniform(-1.5, -0.2)
            m.cheb_shape[i] = (nT, nP)
            m.cheb_range[i] = (300.0, 3000.0, 0.01 * P_ATM, 100.0 * P_ATM)
            cheb += list(a.ravel())
        m.cheb_ptr[i + 1] = len(cheb)
    m.plog = np.array(plog, dtype=float).reshape(-1, 4)
    m.cheb_coef = np.array(cheb, dtype=float)
    fall = [i for i in range(nr) if m.kind[i] in (LINDEMANN, TROE, SRI)]
    for i in rng.permutation(fall)[:int(round(spec.f_chem * len(fall)))]:
        m.chem[i] = True
    rev = [i for i in range(nr) if m.reversible[i]]
    for i in rng.permutation(rev)[:int(round(spec.f_rev_explicit * len(rev)))]:
        m.rev_explicit[i] = True
        m.rev_arr[i] = (m.A[i] * np.exp(rng.uniform(-3.0, 3.0)), m.beta[i] + rng.uniform(-0.5, 0.5),
                        m.Ea[i] + rng.uniform(0.0, 30000.0))


# --------------------------------------------------------------------------
# hand-built tiny mechanisms (tests): every kind, bath-gas cases
# --------------------------------------------------------------------------
def build_mechanism(name, species_comp, reactions, nasa=None, seed=7) -> Mechanism:
    """Mechanism from an explicit reaction list (used for tiny test cases).

    species_comp: list of composition tuples over ELEMENTS (last = bath gas).
    reactions: list of dicts with keys reac, prod (lists of (species, nu)),
      kind, rev, A, beta, Ea and optionally A0, beta0, Ea0, troe (3 or 4
      values), sri (5 values), eff ({species: alpha}), chem (bool),
      rev_arr ((A, beta, Ea) of an explicit reverse rate), plog (list of
      (P [Pa], A, beta, Ea)), cheb (dict with T=(T_min, T_max), P=(P_min,
      P_max) [Pa], coef=[[...]] (N_T x N_P, log10 k)).
    nasa: optional (low [Ns,7], high [Ns,7]); otherwise random smooth fits.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    comp = np.array(species_comp, dtype=np.int64)
    ns, nr = len(comp), len(reactions)
    if nasa is None:
        low = np.zeros((ns, 7))
        high = np.zeros((ns, 7))
        for k in range(ns):
            low[k], high[k], _ = _fit_nasa(rng, comp[k], bath=(k == ns - 1))
    else:
        low, high = (np.array(a, dtype=float) for a in nasa)
    z = lambda: np.zeros(nr)
    m = Mechanism(name=name, species=[_formula(c) for c in comp], composition=comp,
                  W=comp @ ATOMIC_MASS, T_mid=np.full(ns, 1000.0), nasa_low=low, nasa_high=high,
                  kind=np.zeros(nr, dtype=np.int64), reversible=np.zeros(nr, dtype=bool),
                  reac_sp=np.full((nr, MAX_SP), -1, dtype=np.int64),
                  reac_nu=np.zeros((nr, MAX_SP), dtype=np.int64),
                  prod_sp=np.full((nr, MAX_SP), -1, dtype=np.int64),
                  prod_nu=np.zeros((nr, MAX_SP), dtype=np.int64),
                  A=z(), beta=z(), Ea=z(), A0=z(), beta0=z(), Ea0=z(),
                  troe=np.zeros((nr, 4)), troe_n=np.zeros(nr, dtype=np.int64),
                  sri=np.zeros((nr, 5)), eff_ptr=np.zeros(nr + 1, dtype=np.int64),
                  eff_sp=np.zeros(0, dtype=np.int64), eff_val=np.zeros(0))
    eff_sp, eff_val = [], []
    plog, cheb = [], []
    for i, r in enumerate(reactions):
        m.kind[i] = r.get("kind", ELEMENTARY)
        m.chem[i] = bool(r.get("chem", False))
        if "rev_arr" in r:
            m.rev_explicit[i] = True
            m.rev_arr[i] = r["rev_arr"]
        for e in r.get("plog", []):
            plog.append(list(e))
        m.plog_ptr[i + 1] = len(plog)
        if "cheb" in r:
            c = np.array(r["cheb"]["coef"], dtype=float)
            m.cheb_shape[i] = c.shape
            m.cheb_range[i] = list(r["cheb"]["T"]) + list(r["cheb"]["P"])
            cheb += list(c.ravel())
        m.cheb_ptr[i + 1] = len(cheb)
        m.reversible[i] = bool(r.get("rev", True))
        for s, (k, n) in enumerate(r["reac"]):
            m.reac_sp[i, s], m.reac_nu[i, s] = k, n
        for s, (k, n) in enumerate(r["prod"]):
            m.prod_sp[i, s], m.prod_nu[i, s] = k, n
        m.A[i], m.beta[i], m.Ea[i] = r["A"], r.get("beta", 0.0), r.get("Ea", 0.0)
        m.A0[i], m.beta0[i], m.Ea0[i] = r.get("A0", 0.0), r.get("beta0", 0.0), r.get("Ea0", 0.0)
        if "troe" in r:
            t = list(r["troe"])
            m.troe_n[i] = len(t)
            m.troe[i, :len(t)] = t
        if "sri" in r:
            m.sri[i] = r["sri"]
        for k, a in sorted(r.get("eff", {}).items()):
            eff_sp.append(k)
            eff_val.append(a)
        m.eff_ptr[i + 1] = len(eff_sp)
    m.eff_sp = np.array(eff_sp, dtype=np.int64)
    m.eff_val = np.array(eff_val, dtype=float)
    m.plog = np.array(plog, dtype=float).reshape(-1, 4)
    m.cheb_coef = np.array(cheb, dtype=float)
    return m
