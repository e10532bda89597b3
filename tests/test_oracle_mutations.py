"""Planted mistakes: each plausible slip in the oracle's formulas (the source
terms and Jacobian of oracle/kinetics.py, the vector-Jacobian product of
oracle/forms.py) must make at least one pin fail.  The mistake is planted in
a copy of the oracle's source on the CPU; the real oracle is untouched."""
import importlib.util
import math
import os
import types

import numpy as np
import pytest

import synth
from tests import tiny_mechs as tm

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "kinetics.py")
U = 2.0 ** -53


def mutant(old, new):
    src = open(SRC).read()
    assert old in src, old
    mod = types.ModuleType("oracle_mutant")
    exec(compile(src.replace(old, new, 1), "oracle_mutant", "exec"), mod.__dict__)
    return mod


def real():
    return mutant("import numpy as np", "import numpy as np")


# ---- compact pins (each returns True when the pin holds) -------------------
def pin_equilibrium(K, mech):
    rng = np.random.default_rng(1)
    ns = mech.n_species
    T = 1500.0
    _, hrt, sr = K.nasa7(mech, np.array([T]))
    g = (hrt - sr)[:, 0]
    lc0 = math.log(101325.0 / (8314.46261815324 * T))
    target = lc0 - rng.uniform(2.0, 8.0, ns)
    target[-1] = lc0
    w = np.ones(ns)
    w[-1] = 100.0
    lam, *_ = np.linalg.lstsq(mech.composition * w[:, None], (target + g) * w, rcond=None)
    C = np.exp(mech.composition @ lam - g + lc0)
    phi = np.concatenate([[T, 1.0], C[:-1]])[:, None]
    par = np.array([8314.46261815324 * T * C.sum()])
    r = K.rates(mech, 0, phi, par)
    rev = mech.reversible
    return bool(np.all(np.abs(r["Rf"][rev, 0] - r["Rr"][rev, 0]) <= 1e-9 * np.maximum(r["Rf"][rev, 0], r["Rr"][rev, 0])))


def pin_thermo(K, mech):
    T = np.array([700.0, 1500.0])
    cp, hh, ss = K.nasa7(mech, T)
    _, hc, sc = K.nasa7(mech, T + 1e-20j)
    return bool(np.allclose(((T + 1e-20j) * hc).imag / 1e-20, cp, rtol=1e-12)
                and np.allclose(sc.imag / 1e-20, cp / T, rtol=1e-12))


def pin_conservation(K, mech, mode):
    phi, par = synth.make_states(mech, 4, 3, mode)
    f = K.source_terms(mech, mode, phi, par)
    ns = mech.n_species
    ok = True
    for s in range(4):
        def tot(ph):
            T = ph[0]
            V, P = (ph[1], par[s]) if mode == 0 else (par[s], ph[1])
            n = list(ph[2:]) + [P * V / (8314.46261815324 * T) - sum(ph[2:])]
            _, hrt, _ = K.nasa7(mech, T)
            e = hrt if mode == 0 else hrt - 1.0
            return (sum(n[k] * 8314.46261815324 * T * e[k] for k in range(ns)),
                    sum(n[k] * mech.W[k] for k in range(ns)))
        z = phi[:, s].astype(complex) + 1e-30j * f[:, s]
        dE, dm = (x.imag / 1e-30 for x in tot(z))
        E_scale = np.sum(np.abs(8314.46261815324 * phi[0, s] * np.abs(f[2:, s]))) * 1e3 + 1e-300
        m_scale = np.sum(mech.W[:-1] * np.abs(f[2:, s])) + 1e-300
        ok &= abs(dE) <= 1e-9 * E_scale and abs(dm) <= 1e-9 * m_scale
    return bool(ok)


def pin_single_rate(K):
    m = tm.single(dict(reac=[(tm.H, 1), (tm.O2, 1)], prod=[(tm.HO2, 1)], A=7.0, rev=False))
    T, P = 1500.0, 2.0e5
    X = np.zeros(10)
    X[tm.H], X[tm.O2], X[tm.HO2], X[tm.N2] = 0.1, 0.2, 0.05, 0.65
    ntot = P / (8314.46261815324 * T)
    phi = np.concatenate([[T, 1.0], X[:-1] * ntot])[:, None]
    r = K.rates(m, 0, phi, np.array([P]))
    q = 7.0 * (0.1 * ntot) * (0.2 * ntot)
    return bool(abs(r["wdot"][tm.H, 0] + q) <= 1e-12 * q and abs(r["wdot"][tm.HO2, 0] - q) <= 1e-12 * q)


def pin_third_body(K):
    m = tm.single(dict(reac=[(tm.H, 2)], prod=[(tm.H2, 1)], A=2.0, rev=False, kind=synth.THIRD_BODY,
                       eff={tm.H2O: 5.0, tm.N2: 0.5}))
    P, T = 3e5, 1100.0
    ntot = P / (8314.46261815324 * T)
    phi = np.concatenate([[T, 1.0], np.full(9, 0.1 * ntot)])[:, None]
    r = K.rates(m, 0, phi, np.array([P]))
    return bool(abs(r["c"][0, 0] - 0.1 * ntot * (8 + 5.0 + 0.5)) <= 1e-12 * ntot)


def pin_troe_center(K):
    m = tm.single(dict(reac=[(tm.H, 1), (tm.O2, 1)], prod=[(tm.HO2, 1)], A=1e8, rev=False,
                       kind=synth.TROE, A0=1.0, troe=(0.6, 200.0, 1500.0, 4000.0)))
    T = 1200.0
    Fc = 0.4 * math.exp(-T / 200.0) + 0.6 * math.exp(-T / 1500.0) + math.exp(-4000.0 / T)
    F = K.troe_F(m, 0, np.array([T]), np.array([10 ** (0.4 + 0.67 * math.log10(Fc))]))[0]
    return bool(abs(F - Fc) <= 1e-12 * Fc)


def pin_approx(K):
    """Approximate Jacobian (Sec. 3.4): derivatives worked by hand for
    H + H + M -> H2 + M with alpha_N2 = 2, alpha_H2O = 3 (bath gas counted at
    unit efficiency), and pattern superset + tightness on a mechanism whose
    bath gas has non-unit efficiencies."""
    m = tm.single(dict(reac=[(tm.H, 2)], prod=[(tm.H2, 1)], A=1.5e12, beta=-1.1, Ea=0.0, rev=False,
                       kind=synth.THIRD_BODY, eff={tm.N2: 2.0, tm.H2O: 3.0}))
    phi, par = synth.make_states(m, 3, 3, 0)
    Ja = K.jacobian(m, 0, phi, par, form=K.APPROX)
    T, V, P = phi[0], phi[1], par
    C = np.concatenate([phi[2:] / V, (P / (8314.46261815324 * T) - (phi[2:] / V).sum(axis=0))[None]])
    alpha = np.ones(10)
    alpha[tm.N2], alpha[tm.H2O] = 2.0, 3.0
    kf = 1.5e12 * T ** -1.1
    ok = True
    for j in range(9):
        want = -2.0 * kf * (2 * C[tm.H] * (j == tm.H) * (alpha @ C) + C[tm.H] ** 2 * (alpha[j] - 1.0))
        ok &= bool(np.allclose(Ja[2 + tm.H, 2 + j], want, rtol=1e-10, atol=1e-300))
    b = tm.bath_efficiency()
    pa = K.sparsity_pattern(b, K.APPROX)
    phi, par = synth.make_states(b, 12, 4, 0)
    nz = np.any(K.jacobian(b, 0, phi, par, form=K.APPROX) != 0, axis=2)
    forced = np.zeros_like(pa)
    forced[:2, :] = forced[:, :2] = True
    forced[np.arange(11), np.arange(11)] = True
    ok &= not np.any(nz & ~pa) and bool(np.all(nz[pa & ~forced]))
    return bool(ok)


def pin_types(K):
    """P-log at a geometric-mean pressure, a Chebyshev rate against numpy's
    chebval2d, a chemically-activated rate and an explicit reverse rate, each
    worked outside the oracle."""
    R, Rc = 8314.46261815324, 1.98720425864083
    arr = lambda A, b, E, T: A * T ** b * math.exp(-E / (Rc * T))
    ok = True
    T, P = 1100.0, math.sqrt(1.0e4 * 1.0e5)
    ntot = P / (R * T)
    X = np.full(10, 0.1)
    phi = np.concatenate([[T, 1.0], X[:-1] * ntot])[:, None]
    tab = [(1.0e4, 7.0e10, 0.0, 300.0), (1.0e5, 2.0e11, -0.2, 500.0)]
    m = tm.single(dict(reac=[(tm.H, 1), (tm.HO2, 1)], prod=[(tm.OH, 2)], A=1.0, kind=synth.PLOG, plog=tab))
    k = math.sqrt(arr(*tab[0][1:], T) * arr(*tab[1][1:], T))
    ok &= abs(K.rates(m, 0, phi, np.array([P]))["kf"][0, 0] - k) <= 1e-11 * k
    coef = np.array([[9.0, 0.3], [-0.7, 0.1], [0.05, -0.02]])
    m = tm.single(dict(reac=[(tm.OH, 1), (tm.H2, 1)], prod=[(tm.H2O, 1), (tm.H, 1)], A=1.0, kind=synth.CHEB,
                       cheb=dict(T=(300.0, 3000.0), P=(1.0e3, 1.0e7), coef=coef)))
    Tt = (2 / T - 1 / 300.0 - 1 / 3000.0) / (1 / 3000.0 - 1 / 300.0)
    Pt = (2 * math.log10(P) - 3.0 - 7.0) / 4.0
    k = 10.0 ** np.polynomial.chebyshev.chebval2d(Tt, Pt, coef)
    ok &= abs(K.rates(m, 0, phi, np.array([P]))["kf"][0, 0] - k) <= 1e-11 * k
    m = tm.single(dict(reac=[(tm.H, 1), (tm.O2, 1)], prod=[(tm.HO2, 1)], A=5.0e9, beta=0.4, kind=synth.LINDEMANN,
                       chem=True, rev=False, A0=6.0e14, beta0=-1.7, Ea0=500.0))
    k0, kinf = arr(6.0e14, -1.7, 500.0, T), arr(5.0e9, 0.4, 0.0, T)
    Pr = k0 * ntot / kinf
    q = k0 / (1 + Pr) * (0.1 * ntot) ** 2
    ok &= abs(K.rates(m, 0, phi, np.array([P]))["q"][0, 0] - q) <= 1e-11 * q
    m = tm.single(dict(reac=[(tm.H, 1), (tm.O2, 1)], prod=[(tm.OH, 1), (tm.O, 1)], A=2.0e11, beta=-0.3,
                       Ea=15000.0, rev_arr=(1.5e10, 0.1, 800.0)))
    k = arr(1.5e10, 0.1, 800.0, T)
    ok &= abs(K.rates(m, 0, phi, np.array([P]))["kr"][0, 0] - k) <= 1e-11 * k
    return bool(ok)


def all_pins(K, mechs):
    g = mechs("h2co13")
    a = tm.all_kinds()
    return dict(equilibrium=pin_equilibrium(K, g), thermo=pin_thermo(K, g),
                cons_conp=pin_conservation(K, a, 0), cons_conv=pin_conservation(K, a, 1),
                single=pin_single_rate(K), third_body=pin_third_body(K), troe=pin_troe_center(K),
                approx=pin_approx(K), types=pin_types(K))


MUTATIONS = [
    ("lnKc = -dg + dn", "lnKc = dg + dn"),
    ("+ dn * np.log(P_ATM / (R * T))", "- dn * np.log(P_ATM / (R * T))"),
    ("kr[i] = kf[i] * np.exp(-lnKc)", "kr[i] = kf[i] * np.exp(lnKc)"),
    ("np.exp(np.log(A) + beta * np.log(T) - Ea", "np.exp(np.log(A) + beta * np.log(T) + Ea"),
    ("a[2] * T ** 2 / 3 + a[3]", "a[2] * T ** 2 / 2 + a[3]"),
    ("s[k] = a[0] * lnT", "s[k] = a[0] * T"),
    ("+ a[5] / T", "+ a[5] * T"),
    ("(1.0 - mech.W[k] / mech.W[ns - 1]) * wdot[k]", "1.0 * wdot[k]"),
    ("num = sum(E[k] * wdot[k] for k in range(ns))", "num = sum(E[k] * wdot[k] for k in range(ns - 1))"),
    ("Cx = R * (r[\"cp\"] - 1.0)", "Cx = R * r[\"cp\"]"),
    ("wdot[k] = wdot[k] + nu[k, i] * q[i]", "wdot[k] = wdot[k] - nu[k, i] * q[i]"),
    ("a = np.ones(mech.n_species)", "a = np.zeros(mech.n_species)"),
    ("C[ns - 1] = Ctot - acc", "C[ns - 1] = Ctot"),
    ("c = -0.4 - 0.67 * lF", "c = -0.4 - 0.76 * lF"),
    ("f[1] = V * Tdot / T + (R * T * V / P) * Om", "f[1] = V * Tdot / T + (R * V / P) * Om"),
    ("f[1] = P * Tdot / T + R * T * Om", "f[1] = P * Tdot / T + R * Om"),
    # approximate Jacobian (Sec. 3.4)
    ("M = M + (alpha[k] - 1.0) * Cr[k]", "M = M + (alpha[k] - 1.0) * C[k]"),
    ("M = M + (alpha[k] - 1.0) * Cr[k]", "M = M + alpha[k] * Cr[k]"),
    ("        Cr[-1] = _re(C[-1])", "        Cr = _re(C)"),
    ("ref = 1.0 if form == APPROX else a[bath]", "ref = a[bath]"),
    ("    if dense and form != APPROX:", "    if dense:"),
    # less common reaction types
    ("        w = (x - lnPs[m]) / (lnPs[m + 1] - lnPs[m])", "        w = (np.exp(x) - tab[m, 0]) / (tab[m + 1, 0] - tab[m, 0])"),
    ("    Tt = (2.0 / T - 1.0 / Tmin - 1.0 / Tmax) / (1.0 / Tmax - 1.0 / Tmin)", "    Tt = (2.0 * T - Tmin - Tmax) / (Tmax - Tmin)"),
    ("                    cmod[i] = F / (1 + Pr)", "                    cmod[i] = F / (1 + 1 / Pr)"),
    ("        if mech.reversible[i] and mech.rev_explicit[i]:", "        if False:"),
]


# ---- the vector-Jacobian product (oracle/forms.py) -------------------------
FORMS = os.path.join(os.path.dirname(SRC), "forms.py")


def forms_mutant(old, new):
    """oracle.forms with one planted mistake, on the real oracle.kinetics."""
    src = open(FORMS).read()
    assert old in src, old
    src = src.replace(old, new, 1).replace("from .kinetics import", "from oracle.kinetics import")
    mod = types.ModuleType("forms_mutant")
    exec(compile(src, "forms_mutant", "exec"), mod.__dict__)
    return mod


def _y_real(m, mode, phi, par):
    """y = (wdot_0 .. wdot_{Ns-1}, dT/dt) from the real (pinned) rates and
    source terms."""
    import oracle.kinetics as K
    r = K.rates(m, mode, phi, par)
    f, _ = K.source_terms_from_rates(m, mode, r)
    return np.concatenate([r["wdot"], f[:1]], axis=0)


def pin_vjp_state(F, mode):
    """g_Phi against u^T dy/dPhi built from the pinned Jacobian of f (the
    identities of tests/test_oracle_vjp.py)."""
    import oracle.kinetics as K
    m = tm.all_kinds()
    phi, par = synth.make_states(m, 2, 5, mode)
    uw, uT = synth.make_cotangents(m.n_species, 2, 5)
    g, _ = F.vjp(m, mode, phi, par, uw, uT)
    J = K.jacobian(m, mode, phi, par)
    f = K.source_terms(m, mode, phi, par)
    V = phi[1] if mode == 0 else par
    ns = m.n_species
    dw = J[2:] / V
    if mode == 0:
        dw[:, 1] = (J[2:, 1] - f[2:] / V) / V
    dwb = -np.einsum("k,kjn->jn", m.W[:-1] / m.W[-1], dw)
    want = np.einsum("kn,kjn->jn", uw[: ns - 1], dw) + uw[ns - 1] * dwb + uT * J[0]
    scale = np.einsum("kn,kjn->jn", np.abs(uw[: ns - 1]), np.abs(dw)) + np.abs(uw[ns - 1] * dwb) + np.abs(uT * J[0])
    return bool(np.all(np.abs(g - want) <= 1e-8 * scale.max(axis=0) + 1e-300))


def pin_vjp_theta(F, mode):
    """g_theta of one-reaction mechanisms against central differences of
    sum_s u . y (y from the real rates) over copies with ln A, beta or Ea
    moved."""
    H, O, H2, O2, OH, H2O, HO2 = range(7)
    cases = [dict(reac=[(H, 1), (O2, 1)], prod=[(OH, 1), (O, 1)], A=2.0e11, beta=-0.3, Ea=15000.0),
             dict(reac=[(OH, 2)], prod=[(H2, 1), (O2, 1)], A=7.0e10, beta=-0.4, Ea=1200.0, kind=synth.TROE,
                  A0=2.0e12, beta0=-0.8, Ea0=-1500.0, troe=(0.7, 90.0, 1800.0, 5000.0), eff={H2O: 6.0})]
    ok = True
    for rx in cases:
        m = tm.single(rx)
        phi, par = synth.make_states(m, 2, 8, mode)
        uw, uT = synth.make_cotangents(m.n_species, 2, 8)
        _, g = F.vjp(m, mode, phi, par, uw, uT)
        u = np.concatenate([uw, uT[None]], axis=0)
        for p in range(3):
            mp, mm = m.copy(), m.copy()
            d = (1e-5, 1e-6, 1e-6 * max(abs(m.Ea[0]), 100.0))[p]
            if p == 0:
                mp.A[0], mm.A[0] = m.A[0] * math.exp(d), m.A[0] * math.exp(-d)
            elif p == 1:
                mp.beta[0], mm.beta[0] = m.beta[0] + d, m.beta[0] - d
            else:
                mp.Ea[0], mm.Ea[0] = m.Ea[0] + d, m.Ea[0] - d
            dy = (_y_real(mp, mode, phi, par) - _y_real(mm, mode, phi, par)) / (2 * d)
            ok &= bool(abs(g[0, p] - np.sum(u * dy)) <= 1e-6 * np.sum(np.abs(u * dy)))
    return ok


def forms_pins(F):
    return dict(state_conp=pin_vjp_state(F, 0), state_conv=pin_vjp_state(F, 1),
                theta_conp=pin_vjp_theta(F, 0), theta_conv=pin_vjp_theta(F, 1))


FORMS_MUTATIONS = [
    # sign of the dT/dt part of dy/dq
    ("w_q = w_q - (nu.T @ E) * (u_T / aux[\"den\"])", "w_q = w_q + (nu.T @ E) * (u_T / aux[\"den\"])"),
    # the energy-equation denominator dropped
    ("(u_T / aux[\"den\"])[None, :]", "u_T[None, :]"),
    # complex step in Ea not matched by its divisor
    ("Ea=mech.Ea + 1j * hE)", "Ea=mech.Ea + 2j * hE)"),
    # derivative with respect to A instead of ln A
    ("A_c = mech.A * np.exp(1j * hA)", "A_c = mech.A + 1j * hA"),
    # dV/dt (or dP/dt) in place of dT/dt as the last output
    ("np.concatenate([r[\"wdot\"], f[:1]], axis=0)", "np.concatenate([r[\"wdot\"], f[1:2]], axis=0)"),
    # the cotangent of the bath gas dropped from g_Phi
    ("u = np.concatenate([u_wdot, u_T[None, :]], axis=0)        # [Ns+1, n]",
     "u = np.concatenate([u_wdot[:-1], 0 * u_wdot[-1:], u_T[None, :]], axis=0)"),
]


def test_real_forms_pass_vjp_pins():
    res = forms_pins(forms_mutant("import numpy as np", "import numpy as np"))
    assert all(res.values()), res


@pytest.mark.parametrize("old,new", FORMS_MUTATIONS)
def test_planted_vjp_mistake_is_caught(old, new):
    res = forms_pins(forms_mutant(old, new))
    assert not all(res.values()), f"mutation {old!r} -> {new!r} escaped the VJP pins: {res}"


def test_real_oracle_passes_compact_pins(mechs):
    res = all_pins(real(), mechs)
    assert all(res.values()), res


@pytest.mark.parametrize("old,new", MUTATIONS)
def test_planted_mistake_is_caught(mechs, old, new):
    res = all_pins(mutant(old, new), mechs)
    assert not all(res.values()), f"mutation {old!r} -> {new!r} escaped all pins: {res}"
