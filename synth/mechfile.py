"""Plain-text mechanism file format (writer and reader).

One whitespace-separated record per species and per reaction; floating-point
numbers are written with 17 significant digits so that a round trip is exact.

    PJMECH 2
    SPECIES <Ns>
    <name> <W> <T_mid> <nH> <nO> <nC> <nN> <nAr> <low a0..a6> <high a0..a6>
    REACTIONS <Nr>
    <kind> <rev> <n_reac> (<sp> <nu>)* <n_prod> (<sp> <nu>)* <A> <beta> <Ea>
        <A0> <beta0> <Ea0> <troe_n> <a> <T3> <T1> <T2> <sri a b c d e>
        <n_eff> (<sp> <alpha>)*
        <chem> <rev_explicit> <rev A> <rev beta> <rev Ea>
        <n_plog> (<P [Pa]> <A> <beta> <Ea>)*
        <N_T> <N_P> [<T_min> <T_max> <P_min> <P_max> <N_T x N_P log10 k coefficients>]
    END

kind: 0 elementary, 1 third body, 2 Lindemann, 3 Troe, 4 SRI, 5 P-log,
6 Chebyshev.  Species indices are 0-based; the last species is the bath
gas.  Version 1 files end each reaction after the efficiencies.
"""
from __future__ import annotations

import numpy as np

from .mechanism import MAX_SP, Mechanism


def _g(x) -> str:
    return repr(float(x))


def write_mechanism(mech: Mechanism, path: str) -> None:
    lines = ["PJMECH 2", f"SPECIES {mech.n_species}"]
    for k in range(mech.n_species):
        f = [mech.species[k], _g(mech.W[k]), _g(mech.T_mid[k])]
        f += [str(int(c)) for c in mech.composition[k]]
        f += [_g(a) for a in mech.nasa_low[k]] + [_g(a) for a in mech.nasa_high[k]]
        lines.append(" ".join(f))
    lines.append(f"REACTIONS {mech.n_reactions}")
    for i in range(mech.n_reactions):
        r, p = mech.reactants(i), mech.products(i)
        f = [str(int(mech.kind[i])), str(int(bool(mech.reversible[i]))), str(len(r))]
        for k, n in r:
            f += [str(k), str(n)]
        f.append(str(len(p)))
        for k, n in p:
            f += [str(k), str(n)]
        f += [_g(v) for v in (mech.A[i], mech.beta[i], mech.Ea[i], mech.A0[i], mech.beta0[i], mech.Ea0[i])]
        f.append(str(int(mech.troe_n[i])))
        f += [_g(v) for v in mech.troe[i]] + [_g(v) for v in mech.sri[i]]
        eff = mech.efficiencies(i)
        f.append(str(len(eff)))
        for k, a in eff.items():
            f += [str(k), _g(a)]
        f += [str(int(bool(mech.chem[i]))), str(int(bool(mech.rev_explicit[i])))]
        f += [_g(v) for v in mech.rev_arr[i]]
        pl = mech.plog_table(i)
        f.append(str(len(pl)))
        for e in pl:
            f += [_g(v) for v in e]
        nT, nP = (int(x) for x in mech.cheb_shape[i])
        f += [str(nT), str(nP)]
        if nT * nP:
            f += [_g(v) for v in mech.cheb_range[i]] + [_g(v) for v in mech.cheb_table(i).ravel()]
        lines.append(" ".join(f))
    lines.append("END")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")


def read_mechanism(path: str, name: str = "file") -> Mechanism:
    tok = open(path).read().split()
    pos = 0

    def nxt():
        nonlocal pos
        pos += 1
        return tok[pos - 1]

    assert nxt() == "PJMECH", "not a PJMECH file"
    version = int(nxt())
    assert version in (1, 2), "unsupported PJMECH version"
    assert nxt() == "SPECIES"
    ns = int(nxt())
    names, W, Tm, comp, low, high = [], [], [], [], [], []
    for _ in range(ns):
        names.append(nxt())
        W.append(float(nxt()))
        Tm.append(float(nxt()))
        comp.append([int(nxt()) for _ in range(5)])
        low.append([float(nxt()) for _ in range(7)])
        high.append([float(nxt()) for _ in range(7)])
    assert nxt() == "REACTIONS"
    nr = int(nxt())
    kind = np.zeros(nr, dtype=np.int64)
    rev = np.zeros(nr, dtype=bool)
    rsp = np.full((nr, MAX_SP), -1, dtype=np.int64)
    rnu = np.zeros((nr, MAX_SP), dtype=np.int64)
    psp = np.full((nr, MAX_SP), -1, dtype=np.int64)
    pnu = np.zeros((nr, MAX_SP), dtype=np.int64)
    fl = np.zeros((nr, 6))
    troe = np.zeros((nr, 4))
    troe_n = np.zeros(nr, dtype=np.int64)
    sri = np.zeros((nr, 5))
    eff_ptr, eff_sp, eff_val = [0], [], []
    chem = np.zeros(nr, dtype=bool)
    rev_explicit = np.zeros(nr, dtype=bool)
    rev_arr = np.zeros((nr, 3))
    plog_ptr, plog = [0], []
    cheb_ptr, cheb_shape, cheb_range, cheb_coef = [0], np.zeros((nr, 2), dtype=np.int64), np.zeros((nr, 4)), []
    for i in range(nr):
        kind[i] = int(nxt())
        rev[i] = bool(int(nxt()))
        for sp, nu in ((rsp, rnu), (psp, pnu)):
            m = int(nxt())
            for s in range(m):
                sp[i, s] = int(nxt())
                nu[i, s] = int(nxt())
        fl[i] = [float(nxt()) for _ in range(6)]
        troe_n[i] = int(nxt())
        troe[i] = [float(nxt()) for _ in range(4)]
        sri[i] = [float(nxt()) for _ in range(5)]
        for _ in range(int(nxt())):
            eff_sp.append(int(nxt()))
            eff_val.append(float(nxt()))
        eff_ptr.append(len(eff_sp))
        if version >= 2:
            chem[i] = bool(int(nxt()))
            rev_explicit[i] = bool(int(nxt()))
            rev_arr[i] = [float(nxt()) for _ in range(3)]
            for _ in range(int(nxt())):
                plog.append([float(nxt()) for _ in range(4)])
            nT, nP = int(nxt()), int(nxt())
            cheb_shape[i] = (nT, nP)
            if nT * nP:
                cheb_range[i] = [float(nxt()) for _ in range(4)]
                cheb_coef += [float(nxt()) for _ in range(nT * nP)]
        plog_ptr.append(len(plog))
        cheb_ptr.append(len(cheb_coef))
    assert nxt() == "END"
    return Mechanism(name=name, species=names, composition=np.array(comp, dtype=np.int64),
                     W=np.array(W), T_mid=np.array(Tm), nasa_low=np.array(low), nasa_high=np.array(high),
                     kind=kind, reversible=rev, reac_sp=rsp, reac_nu=rnu, prod_sp=psp, prod_nu=pnu,
                     A=fl[:, 0].copy(), beta=fl[:, 1].copy(), Ea=fl[:, 2].copy(),
                     A0=fl[:, 3].copy(), beta0=fl[:, 4].copy(), Ea0=fl[:, 5].copy(),
                     troe=troe, troe_n=troe_n, sri=sri,
                     eff_ptr=np.array(eff_ptr, dtype=np.int64), eff_sp=np.array(eff_sp, dtype=np.int64),
                     eff_val=np.array(eff_val, dtype=float), chem=chem, rev_explicit=rev_explicit,
                     rev_arr=rev_arr, plog_ptr=np.array(plog_ptr, dtype=np.int64),
                     plog=np.array(plog, dtype=float).reshape(-1, 4),
                     cheb_ptr=np.array(cheb_ptr, dtype=np.int64), cheb_shape=cheb_shape, cheb_range=cheb_range,
                     cheb_coef=np.array(cheb_coef, dtype=float))
