"""Pins of the oracle's less common reaction types (named in Sec. 2.2 and
Sec. 3.2 without their formulas; the standard published forms): P-log,
Chebyshev, chemically-activated falloff and explicit reverse Arrhenius
parameters -- values worked by hand or by a library routine, limits,
conservation, and the complex-step Jacobian against central differences."""
import numpy as np
import pytest

import oracle
import synth
from tests import tiny_mechs as tm
from tests.tiny_mechs import H, O, H2, O2, OH, H2O, HO2, N2

R = 8314.46261815324
R_CAL = 1.98720425864083


def _arr(A, b, Ea, T):
    T = np.longdouble(T)
    return np.longdouble(A) * T ** np.longdouble(b) * np.exp(-np.longdouble(Ea) / (np.longdouble(R_CAL) * T))


def _state(m, T, P, X=None):
    """One CONP state with temperature T, pressure P and mole fractions X."""
    ns = m.n_species
    if X is None:
        X = np.full(ns, 1.0 / ns)
    ntot = P / (R * T)
    phi = np.concatenate([[T, 1.0], X[:-1] * ntot])[:, None]
    return phi, np.array([P])


PLOG_TAB = [(1.0e4, 7.0e10, 0.0, 300.0), (1.0e5, 2.0e11, -0.2, 500.0), (1.0e6, 9.0e11, -0.5, 900.0)]


def _plog_mech():
    return tm.single(dict(reac=[(H, 1), (HO2, 1)], prod=[(OH, 2)], A=1.0, kind=synth.PLOG, plog=PLOG_TAB))


@pytest.mark.parametrize("T", [700.0, 1900.0])
def test_plog_at_tabulated_pressures_and_between(T):
    m = _plog_mech()
    ks = [float(_arr(A, b, Ea, T)) for _, A, b, Ea in PLOG_TAB]
    for (P, *_), k in zip(PLOG_TAB, ks):
        kf = oracle.rates(m, 0, *_state(m, T, P))["kf"][0, 0]
        assert abs(kf - k) <= 1e-13 * k
    for a in range(2):                      # geometric mean pressure: geometric mean rate
        P = np.sqrt(PLOG_TAB[a][0] * PLOG_TAB[a + 1][0])
        kf = oracle.rates(m, 0, *_state(m, T, P))["kf"][0, 0]
        assert abs(kf - np.sqrt(ks[a] * ks[a + 1])) <= 1e-12 * kf
    for P, k in ((10.0, ks[0]), (1.0e9, ks[-1])):   # held at the end values outside the table
        kf = oracle.rates(m, 0, *_state(m, T, P))["kf"][0, 0]
        assert abs(kf - k) <= 1e-13 * k
    # continuous across an inner pressure
    P1 = PLOG_TAB[1][0]
    lo = oracle.rates(m, 0, *_state(m, T, P1 * (1 - 1e-9)))["kf"][0, 0]
    hi = oracle.rates(m, 0, *_state(m, T, P1 * (1 + 1e-9)))["kf"][0, 0]
    assert abs(lo - hi) <= 1e-7 * lo


def test_chebyshev_against_numpy_chebval2d():
    rng = np.random.default_rng(4)
    coef = rng.standard_normal((4, 3)) * np.array([[2.0], [0.5], [0.2], [0.05]])
    coef[0, 0] += 9.0
    Tmin, Tmax, Pmin, Pmax = 300.0, 3000.0, 1.0e3, 1.0e7
    m = tm.single(dict(reac=[(OH, 1), (H2, 1)], prod=[(H2O, 1), (H, 1)], A=1.0, kind=synth.CHEB,
                       cheb=dict(T=(Tmin, Tmax), P=(Pmin, Pmax), coef=coef)))
    for T, P in ((350.0, 2.0e3), (1234.5, 3.3e5), (2900.0, 8.0e6), (1000.0, 1.0e5)):
        Tt = (2 / T - 1 / Tmin - 1 / Tmax) / (1 / Tmax - 1 / Tmin)
        Pt = (2 * np.log10(P) - np.log10(Pmin) - np.log10(Pmax)) / (np.log10(Pmax) - np.log10(Pmin))
        ref = 10.0 ** np.polynomial.chebyshev.chebval2d(Tt, Pt, coef)
        kf = oracle.rates(m, 0, *_state(m, T, P))["kf"][0, 0]
        assert abs(kf - ref) <= 1e-12 * ref


def test_chebyshev_two_terms_at_the_range_ends():
    """log10 k = a0 + a1 T~ with T~ = -1 at T_min and +1 at T_max."""
    m = tm.single(dict(reac=[(OH, 1), (H2, 1)], prod=[(H2O, 1), (H, 1)], A=1.0, kind=synth.CHEB,
                       cheb=dict(T=(500.0, 2500.0), P=(1e4, 1e6), coef=[[9.0], [0.4]])))
    for T, ref in ((500.0, 10 ** 8.6), (2500.0, 10 ** 9.4)):
        kf = oracle.rates(m, 0, *_state(m, T, 5e4))["kf"][0, 0]
        assert abs(kf - ref) <= 1e-12 * ref


def test_chemically_activated_by_hand_and_limits():
    """Lindemann chemically-activated H + O2 (+M) -> HO2 (the product side
    irrelevant here, irreversible): q = k0 / (1 + Pr) C_H C_O2, Pr = k0 [M] / k_inf."""
    A, b, Ea, A0, b0, Ea0 = 5.0e9, 0.4, 0.0, 6.0e14, -1.7, 500.0
    m = tm.single(dict(reac=[(H, 1), (O2, 1)], prod=[(HO2, 1)], A=A, beta=b, Ea=Ea, kind=synth.LINDEMANN,
                       chem=True, rev=False, A0=A0, beta0=b0, Ea0=Ea0))
    T = 1300.0
    X = np.full(10, 0.05)
    X[N2] = 1 - 0.45
    for P in (1.0e3, 1.0e5, 1.0e8):
        phi, par = _state(m, T, P, X)
        ntot = P / (R * T)
        k0, kinf = float(_arr(A0, b0, Ea0, T)), float(_arr(A, b, Ea, T))
        Pr = k0 * ntot / kinf
        q = k0 / (1 + Pr) * (0.05 * ntot) ** 2
        got = oracle.rates(m, 0, phi, par)["q"][0, 0]
        assert abs(got - q) <= 1e-12 * q
    # high-pressure limit: k0 / (1 + Pr) -> k_inf / [M]
    phi, par = _state(m, T, 1.0e14, X)
    ntot = 1.0e14 / (R * T)
    got = oracle.rates(m, 0, phi, par)["q"][0, 0] / (0.05 * ntot) ** 2
    assert abs(got - float(_arr(A, b, Ea, T)) / ntot) <= 1e-4 * got


def test_explicit_reverse_rate_by_hand():
    Ar, br, Ear = 1.5e10, 0.1, 800.0
    m = tm.single(dict(reac=[(H, 1), (O2, 1)], prod=[(OH, 1), (O, 1)], A=2.0e11, beta=-0.3, Ea=15000.0,
                       rev_arr=(Ar, br, Ear)))
    T = 1700.0
    phi, par = _state(m, T, 2.0e5)
    r = oracle.rates(m, 0, phi, par)
    kr = float(_arr(Ar, br, Ear, T))
    assert abs(r["kr"][0, 0] - kr) <= 1e-13 * kr
    C = r["C"][:, 0]
    assert abs(r["Rr"][0, 0] - kr * C[OH] * C[O]) <= 1e-13 * r["Rr"][0, 0]


@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
def test_all_types_conserve_elements_and_mass(mode):
    m = tm.all_types()
    phi, par = synth.make_states(m, 16, 7, mode)
    r = oracle.rates(m, mode, phi, par)
    w = r["wdot"]
    for e in range(m.composition.shape[1]):
        a = m.composition[:, e][:, None]
        assert np.all(np.abs((a * w).sum(axis=0)) <= 64 * 2.0 ** -53 * np.abs(a * w).sum(axis=0) + 1e-300)
    mw = m.W[:, None] * w
    assert np.all(np.abs(mw.sum(axis=0)) <= 64 * 2.0 ** -53 * np.abs(mw).sum(axis=0))


@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
def test_all_types_complex_step_jacobian_against_central_differences(mode):
    m = tm.all_types()
    phi, par = synth.make_states(m, 6, 8, mode)
    J = oracle.jacobian(m, mode, phi, par)
    _, env = oracle.jacobian_envelope(m, mode, phi, par)
    f0 = oracle.source_terms(m, mode, phi, par)
    for j in range(phi.shape[0]):
        h = 1e-6 * np.abs(phi[j])
        p1, p2 = phi.copy(), phi.copy()
        p1[j] += h
        p2[j] -= h
        fd = (oracle.source_terms(m, mode, p1, par) - oracle.source_terms(m, mode, p2, par)) / (2 * h)
        tol = 1e-5 * env[:, j] + 1e-12 * np.abs(f0).max(axis=0) / h
        assert np.all(np.abs(fd - J[:, j]) <= tol), (j, float(np.max(np.abs(fd - J[:, j]) / tol)))
