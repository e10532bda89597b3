"""Pins of the CPU oracle to facts outside itself (closed forms, conservation
laws, a computed chemical equilibrium, finite differences).  CPU only."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import kinetics as K
from tests import tiny_mechs as tm

U = 2.0 ** -53


def one_state(mech, T, P, X, V=1.0, mode=synth.CONP):
    """State from mole fractions X (all species, last = bath gas)."""
    X = np.asarray(X, float) / np.sum(X)
    ntot = P * V / (K.R * T)
    phi = np.empty((mech.n_species + 1, 1))
    phi[0, 0] = T
    phi[1, 0] = V if mode == synth.CONP else P
    phi[2:, 0] = X[:-1] * ntot
    param = np.array([P if mode == synth.CONP else V])
    return phi, param


# ---------------------------------------------------------------- thermo ----
def test_nasa7_constant_cp_closed_form():
    """cp/R = a0, h/RT = a0 + a5/T, s/R = a0 ln T + a6 for a constant-cp species."""
    low, high = tm.constant_cp_nasa(10, cp_R=3.5, a5=-1234.0, a6=5.5)
    m = synth.build_mechanism("c", tm.SP, [dict(reac=[(0, 1), (3, 1)], prod=[(4, 1), (1, 1)], A=1.0)],
                              nasa=(low, high))
    T = np.array([700.0, 1300.0, 2400.0])
    cp, h, s = K.nasa7(m, T)
    assert np.allclose(cp, 3.5, rtol=0, atol=1e-15)
    assert np.allclose(h, 3.5 - 1234.0 / T, rtol=1e-15)
    assert np.allclose(s, 3.5 * np.log(T) + 5.5, rtol=1e-15)


@pytest.mark.parametrize("name", ["h2co13", "gri53"])
def test_nasa7_thermodynamic_consistency(mechs, name):
    """dH/dT = Cp and dS/dT = Cp/T in both ranges (complex-step in T)."""
    m = mechs(name)
    T = np.array([650.0, 900.0, 1200.0, 2300.0])
    h = 1e-20
    cp, hh, ss = K.nasa7(m, T)
    _, hc, sc = K.nasa7(m, T + 1j * h)
    dH = ((T + 1j * h) * hc).imag / h           # d(h/R)/dT  with h/R = T * (h/RT)
    dS = sc.imag / h
    assert np.allclose(dH, cp, rtol=1e-12)
    assert np.allclose(dS, cp / T, rtol=1e-12)


def test_nasa7_continuity_at_T_mid(mechs):
    """The generator makes h and s continuous at T_mid; both ranges agree there."""
    m = mechs("gri53")
    Tm = m.T_mid[0]
    _, h_hi, s_hi = K.nasa7(m, np.array([Tm]))
    _, h_lo, s_lo = K.nasa7(m, np.array([np.nextafter(Tm, 0)]))
    assert np.allclose(h_hi, h_lo, rtol=1e-9, atol=1e-9)
    assert np.allclose(s_hi, s_lo, rtol=1e-9, atol=1e-9)


# ----------------------------------------------------------- rate laws ----
def test_arrhenius_closed_forms():
    assert K.arrhenius(3.0, 1.0, 0.0, 1000.0) == pytest.approx(3000.0, rel=1e-15)
    # Ea = R_cal T ln 2 halves the rate
    T = 1234.0
    assert K.arrhenius(5.0, 0.0, K.R_CAL * T * math.log(2.0), T) == pytest.approx(2.5, rel=1e-14)
    assert K.arrhenius(1.0, -2.0, 0.0, 10.0) == pytest.approx(0.01, rel=1e-15)


def test_single_irreversible_rate_by_hand():
    """A + B -> C: wdot = (-k CA CB, -k CA CB, +k CA CB), k = A exactly."""
    m = tm.single(dict(reac=[(tm.H, 1), (tm.O2, 1)], prod=[(tm.HO2, 1)], A=7.0, rev=False))
    T, P = 1500.0, 2.0e5
    X = np.zeros(10)
    X[tm.H], X[tm.O2], X[tm.HO2], X[tm.N2] = 0.1, 0.2, 0.05, 0.65
    phi, par = one_state(m, T, P, X)
    r = K.rates(m, synth.CONP, phi, par)
    Ctot = P / (K.R * T)
    q = 7.0 * (0.1 * Ctot) * (0.2 * Ctot)
    assert r["wdot"][tm.H, 0] == pytest.approx(-q, rel=1e-13)
    assert r["wdot"][tm.O2, 0] == pytest.approx(-q, rel=1e-13)
    assert r["wdot"][tm.HO2, 0] == pytest.approx(q, rel=1e-13)
    assert np.all(r["wdot"][[tm.O, tm.H2, tm.OH, tm.H2O, tm.N, tm.NO, tm.N2], 0] == 0)


def test_stoichiometric_powers():
    """2 OH -> H2O + O uses C_OH squared."""
    m = tm.single(dict(reac=[(tm.OH, 2)], prod=[(tm.O, 1), (tm.H2O, 1)], A=3.0, rev=False))
    X = np.zeros(10)
    X[tm.OH], X[tm.N2] = 0.3, 0.7
    phi, par = one_state(m, 1000.0, 101325.0, X)
    r = K.rates(m, synth.CONP, phi, par)
    C = 0.3 * 101325.0 / (K.R * 1000.0)
    assert r["wdot"][tm.OH, 0] == pytest.approx(-2 * 3.0 * C * C, rel=1e-13)
    assert r["wdot"][tm.O, 0] == pytest.approx(3.0 * C * C, rel=1e-13)


def test_third_body_unit_efficiencies_is_total_concentration():
    m = tm.single(dict(reac=[(tm.H, 2)], prod=[(tm.H2, 1)], A=2.0, rev=False, kind=synth.THIRD_BODY))
    X = np.full(10, 0.1)
    phi, par = one_state(m, 1100.0, 3e5, X)
    r = K.rates(m, synth.CONP, phi, par)
    assert r["c"][0, 0] == pytest.approx(3e5 / (K.R * 1100.0), rel=1e-14)


def test_third_body_efficiencies_weight_concentrations():
    m = tm.single(dict(reac=[(tm.H, 2)], prod=[(tm.H2, 1)], A=2.0, rev=False, kind=synth.THIRD_BODY,
                       eff={tm.H2O: 5.0, tm.N2: 0.5, tm.O2: 0.0}))
    X = np.full(10, 0.1)
    phi, par = one_state(m, 1100.0, 3e5, X)
    r = K.rates(m, synth.CONP, phi, par)
    Ci = 0.1 * 3e5 / (K.R * 1100.0)
    assert r["c"][0, 0] == pytest.approx(Ci * (7 + 5.0 + 0.5 + 0.0), rel=1e-13)


def _falloff_mech(kind, A0, extra):
    d = dict(reac=[(tm.H, 1), (tm.O2, 1)], prod=[(tm.HO2, 1)], A=1e8, beta=0.5, Ea=1000.0,
             rev=False, kind=kind, A0=A0, beta0=-1.0, Ea0=200.0)
    d.update(extra)
    return tm.single(d)


def _c(m, T=1200.0, P=2e5):
    X = np.full(10, 0.1)
    phi, par = one_state(m, T, P, X)
    r = K.rates(m, synth.CONP, phi, par)
    return r


def test_lindemann_limits():
    """Pr -> 0: c -> Pr (rate k0 [M]); Pr -> inf: c -> 1 (rate k_inf)."""
    lo = _c(_falloff_mech(synth.LINDEMANN, 1e-30, {}))
    T = 1200.0
    M = 2e5 / (K.R * T)
    k0 = 1e-30 * T ** -1.0 * math.exp(-200.0 / (K.R_CAL * T))
    kinf = 1e8 * T ** 0.5 * math.exp(-1000.0 / (K.R_CAL * T))
    assert lo["c"][0, 0] == pytest.approx(k0 * M / kinf, rel=1e-12)
    hi = _c(_falloff_mech(synth.LINDEMANN, 1e40, {}))
    assert hi["c"][0, 0] == pytest.approx(1.0, rel=1e-12)


def test_troe_reduces_to_lindemann():
    """a = 0 and T3 -> inf give Fcent = 1, hence F = 1 (3-parameter form)."""
    lind = _c(_falloff_mech(synth.LINDEMANN, 1e12, {}))
    troe = _c(_falloff_mech(synth.TROE, 1e12, dict(troe=(0.0, 1e300, 1000.0))))
    assert troe["c"][0, 0] == pytest.approx(lind["c"][0, 0], rel=1e-14)


def test_troe_center_of_falloff_curve():
    """At log10 Pr = 0.4 + 0.67 log10 Fcent the Troe form returns F = Fcent."""
    m = _falloff_mech(synth.TROE, 1.0, dict(troe=(0.6, 200.0, 1500.0, 4000.0)))
    T = 1200.0
    Fcent = 0.4 * math.exp(-T / 200.0) + 0.6 * math.exp(-T / 1500.0) + math.exp(-4000.0 / T)
    Pr = 10 ** (0.4 + 0.67 * math.log10(Fcent))
    F = K.troe_F(m, 0, np.array([T]), np.array([Pr]))
    assert F[0] == pytest.approx(Fcent, rel=1e-13)
    # far from the centre the curve flattens towards Fcent^(1/(1+1/0.14^2))
    F_far = K.troe_F(m, 0, np.array([T]), np.array([1e300]))
    assert F_far[0] == pytest.approx(Fcent ** (1 / (1 + 1 / 0.14 ** 2)), rel=5e-3)


def test_sri_reduces_to_lindemann_and_unit_pr():
    lind = _c(_falloff_mech(synth.LINDEMANN, 1e12, {}))
    sri = _c(_falloff_mech(synth.SRI, 1e12, dict(sri=(0.0, 1.0, 1e300, 1.0, 0.0))))
    assert sri["c"][0, 0] == pytest.approx(lind["c"][0, 0], rel=1e-14)
    # Pr = 1: X = 1 so F = d (a exp(-b/T) + exp(-T/c)) T^e
    m = _falloff_mech(synth.SRI, 1.0, dict(sri=(0.5, 300.0, 900.0, 1.2, 0.3)))
    T = 1500.0
    F = K.sri_F(m, 0, np.array([T]), np.array([1.0]))
    assert F[0] == pytest.approx(1.2 * (0.5 * math.exp(-300 / T) + math.exp(-T / 900.0)) * T ** 0.3,
                                 rel=1e-14)


# ------------------------------------------------- conservation laws ----
@pytest.mark.parametrize("name", ["h2co13", "gri53", "gri53_types", "usc111"])
def test_element_and_mass_conservation(mechs, name):
    m = mechs(name)
    phi, par = synth.make_states(m, 64, 5, synth.CONP)
    r = K.rates(m, synth.CONP, phi, par)
    w = r["wdot"]
    a = m.composition.T.astype(float)              # [Ne, Ns]
    bal = a @ w
    scale = np.abs(a) @ np.abs(w)
    assert np.all(np.abs(bal) <= 64 * U * scale + 1e-300)
    mass = m.W @ w
    assert np.all(np.abs(mass) <= 64 * U * (np.abs(m.W) @ np.abs(w)))


@pytest.mark.parametrize("name", ["h2co13", "gri53", "gri53_types"])
def test_conp_conv_share_production_rates(mechs, name):
    m = mechs(name)
    pc, parc = synth.make_states(m, 32, 9, synth.CONP)
    pv, parv = synth.make_states(m, 32, 9, synth.CONV)
    wc = K.rates(m, synth.CONP, pc, parc)["wdot"]
    wv = K.rates(m, synth.CONV, pv, parv)["wdot"]
    _, env = K.source_term_envelope(m, synth.CONP, pc, parc)
    V = pc[1]
    assert np.all(np.abs(wc - wv)[:-1] <= 1e-12 * env[2:] / V)


def _directional(fun, phi, direction, h=1e-30):
    return fun(phi.astype(complex) + 1j * h * direction).imag / h


@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
@pytest.mark.parametrize("name", ["h2co13", "gri53", "gri53_types"])
def test_energy_and_mass_conserved_along_source_terms(mechs, name, mode):
    """Adiabatic closed system: total enthalpy (CONP) or internal energy (CONV)
    and total mass, with the bath gas from the ideal-gas law, are constant
    along f (Sec. 2.2)."""
    m = mechs(name)
    phi, par = synth.make_states(m, 16, 3, mode)
    f = K.source_terms(m, mode, phi, par)
    ns = m.n_species

    def totals(ph, pr):
        T = ph[0]
        if mode == synth.CONP:
            V, P = ph[1], pr
        else:
            P, V = ph[1], pr
        n = list(ph[2:])
        n.append(P * V / (K.R * T) - sum(ph[2:]))
        _, hrt, _ = K.nasa7(m, T)
        e = hrt if mode == synth.CONP else hrt - 1.0
        E = sum(n[k] * K.R * T * e[k] for k in range(ns))
        mass = sum(n[k] * m.W[k] for k in range(ns))
        return np.stack([E, mass])

    d = np.stack([_directional(lambda p: totals(p, par[s:s + 1])[0], phi[:, s:s + 1], f[:, s:s + 1])
                  for s in range(16)])
    dm = np.stack([_directional(lambda p: totals(p, par[s:s + 1])[1], phi[:, s:s + 1], f[:, s:s + 1])
                   for s in range(16)])
    # scale: sum of magnitudes of the individual contributions
    r = K.rates(m, mode, phi, par)
    e = r["h"] if mode == synth.CONP else r["h"] - 1.0
    _, env = K.source_term_envelope(m, mode, phi, par)
    escale = np.sum(np.abs(K.R * phi[0] * e[:-1]) * env[2:], axis=0) * 4
    mscale = np.sum(m.W[:-1, None] * env[2:], axis=0) * 4
    assert np.all(np.abs(d[:, 0]) <= 1e-11 * escale + 1e-300)
    assert np.all(np.abs(dm[:, 0]) <= 1e-11 * mscale + 1e-300)


# ---------------------------------------------------- equilibrium ----
@pytest.mark.parametrize("name", ["h2co13", "gri53", "usc111"])
def test_rates_balance_at_computed_equilibrium(mechs, name):
    """C_k = (P_atm/RT) exp(sum_e a_ek lambda_e - g_k/RT) is the ideal-gas
    Gibbs-minimum composition for element potentials lambda; there every
    reversible element-balanced reaction has equal forward and reverse rates."""
    m = mechs(name)
    rng = np.random.default_rng(4)
    ns = m.n_species
    for T in (800.0, 1400.0, 2200.0):
        cp, hrt, sr = K.nasa7(m, np.array([T]))
        g = (hrt - sr)[:, 0]
        # element potentials by weighted least squares so that every ln C_k is
        # near a moderate target and the bath gas dominates the mixture
        lc0 = math.log(K.P_ATM / (K.R * T))
        target = lc0 - rng.uniform(2.0, 12.0, ns)
        target[-1] = lc0
        w = np.ones(ns)
        w[-1] = 100.0
        lam, *_ = np.linalg.lstsq(m.composition * w[:, None], (target + g) * w, rcond=None)
        C = np.exp(m.composition @ lam - g) * (K.P_ATM / (K.R * T))
        phi = np.empty((ns + 1, 1))
        phi[0], phi[1] = T, 1.0
        phi[2:, 0] = C[:-1]
        par = np.array([K.R * T * C.sum()])
        r = K.rates(m, synth.CONP, phi, par)
        rev = m.reversible
        Rf, Rr = r["Rf"][rev, 0], r["Rr"][rev, 0]
        # the bath gas comes from C_tot - sum C_k: its relative rounding error is
        # about u * C_tot / C_Ns, inherited by the reactions it takes part in
        kappa = C.sum() / C[-1]
        bath = np.array([any(k == ns - 1 for k, _ in m.reactants(i) + m.products(i))
                         for i in np.flatnonzero(rev)])
        tol = 1e-11 + np.where(bath, 64 * U * kappa, 0.0)
        assert np.all(np.abs(Rf - Rr) <= tol * np.maximum(Rf, Rr))


def test_wrong_equilibrium_sign_would_fail(mechs):
    """The equilibrium pin detects a flipped Gibbs-energy sign (planted in a
    copy of the oracle's formula on the CPU)."""
    m = mechs("h2co13")
    T = 1400.0
    cp, hrt, sr = K.nasa7(m, np.array([T]))
    g = (hrt - sr)[:, 0]
    C = np.exp(m.composition @ np.array([0.1, -0.2, 0.3, (g[-1] + 3.0) / 2.0, 0.0]) - g) * (K.P_ATM / (K.R * T))
    nu = K.net_stoich(m)
    i = int(np.flatnonzero(m.reversible)[0])
    good = np.exp(-(nu[:, i] @ g)) * (K.P_ATM / (K.R * T)) ** nu[:, i].sum()
    bad = np.exp(+(nu[:, i] @ g)) * (K.P_ATM / (K.R * T)) ** nu[:, i].sum()
    ratio = np.prod(C ** nu[:, i])
    assert ratio == pytest.approx(good, rel=1e-11)
    assert abs(ratio / bad - 1) > 1e-3


# ----------------------------------------------------------- Jacobian ----
def test_jacobian_closed_form_first_order():
    """A -> B irreversible, CONV: J[A,A] = -k, J[B,A] = +k, J[A,T] = -n_A k (beta + theta/T)/T."""
    A, beta, Ea = 3.0e6, 0.7, 9000.0
    m = tm.single(dict(reac=[(tm.HO2, 1)], prod=[(tm.H, 1), (tm.O2, 1)], A=A, beta=beta, Ea=Ea,
                       rev=False))
    X = np.zeros(10)
    X[tm.HO2], X[tm.N2] = 0.2, 0.8
    T = 1300.0
    phi, par = one_state(m, T, 1.5e5, X, V=2.0, mode=synth.CONV)
    J = K.jacobian(m, synth.CONV, phi, par)[:, :, 0]
    k = A * T ** beta * math.exp(-Ea / (K.R_CAL * T))
    nA = phi[2 + tm.HO2, 0]
    iA, iH = 2 + tm.HO2, 2 + tm.H
    assert J[iA, iA] == pytest.approx(-k, rel=1e-13)
    assert J[iH, iA] == pytest.approx(k, rel=1e-13)
    assert J[iA, 0] == pytest.approx(-nA * k * (beta + Ea / K.R_CAL / T) / T, rel=1e-12)
    assert J[iA, 1] == 0.0  # CONV: d/dP of n_A/V is zero


@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
@pytest.mark.parametrize("mk", ["all_kinds", "bath_efficiency", "h2co13", "gri53", "gri53_types"])
def test_jacobian_matches_central_differences(mechs, mk, mode):
    m = getattr(tm, mk)() if mk in ("all_kinds", "bath_efficiency", "all_types") else mechs(mk)
    # no vanishing mole fractions, so a relative step of 1e-6 balances the
    # O(h^2) truncation against the O(u/h) rounding of the difference
    phi, par = synth.make_states(m, 6, 17, mode, alpha=5.0)
    J, env = K.jacobian_envelope(m, mode, phi, par)
    _, envf = K.source_term_envelope(m, mode, phi, par)
    N = m.n_species + 1
    for j in range(N):
        h = 1e-6 * np.abs(phi[j])
        p1, p2 = phi.copy(), phi.copy()
        p1[j] += h
        p2[j] -= h
        fd = (K.source_terms(m, mode, p1, par) - K.source_terms(m, mode, p2, par)) / (2 * h)
        err = np.abs(fd - J[:, j])
        # truncation O(h^2) relative to the entry's envelope, plus the
        # difference quotient's own rounding, u * (sum of |terms| of f) / h
        tol = 1e-4 * env[:, j] + 16 * U * envf / h
        assert np.all(err <= tol), (j, np.max(err / tol))


@pytest.mark.parametrize("mk", ["all_kinds", "bath_efficiency", "all_types", "h2co13", "gri53", "gri53_types"])
def test_pattern_superset_and_tight(mechs, mk):
    m = getattr(tm, mk)() if mk in ("all_kinds", "bath_efficiency", "all_types") else mechs(mk)
    mask = K.sparsity_pattern(m)
    phi, par = synth.make_states(m, 24, 23, synth.CONP)
    J = K.jacobian(m, synth.CONP, phi, par)
    nz = (J != 0).any(axis=2)
    assert not np.any(nz & ~mask), "complex-step nonzero outside the pattern"
    forced = np.zeros_like(mask)
    forced[:2, :] = forced[:, :2] = True
    forced[np.arange(len(mask)), np.arange(len(mask))] = True
    assert not np.any(mask & ~forced & ~nz), "pattern entry never nonzero"


def test_bath_gas_rules_make_rows_dense():
    """Sec. 3.4: a bath-gas reactant, or a non-unit bath-gas efficiency, fills
    every species row the reaction changes."""
    m = tm.bath_efficiency()
    mask = K.sparsity_pattern(m)
    for sp in (tm.O, tm.O2, tm.H, tm.HO2):
        assert mask[2 + sp, 2:].all()
    m2 = tm.all_kinds()
    mask2 = K.sparsity_pattern(m2)
    for sp in (tm.N, tm.NO, tm.O):          # N + NO -> N2 + O
        assert mask2[2 + sp, 2:].all()


def test_csr_csc_are_transposes(mechs):
    m = mechs("gri53")
    rp, ci = K.csr_pattern(m)
    cp_, ri = K.csc_pattern(m)
    N = m.n_species + 1
    A = np.zeros((N, N), dtype=bool)
    A[np.repeat(np.arange(N), np.diff(rp)), ci] = True
    B = np.zeros((N, N), dtype=bool)
    B[ri, np.repeat(np.arange(N), np.diff(cp_))] = True
    assert (A == B).all() and A.sum() == len(ci) == len(ri)
    for i in range(N):
        assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0)
