"""Pins of the oracle's approximate Jacobian (Sec. 3.4, "Sparsity patterns"):
the derivatives that reach a rate of progress through the bath-gas
concentration, and those that a non-unit bath-gas efficiency spreads over
every species, are left out.  Checked against derivatives worked out by hand
on one-reaction mechanisms, against the exact form where the bath gas takes
no part, through the structure of what is dropped, and on the pattern."""
import numpy as np
import pytest

import oracle
import synth
from oracle import kinetics as K
from tests import tiny_mechs as tm
from tests.tiny_mechs import H, O, H2, O2, OH, H2O, N, NO, N2

R = 8314.46261815324
R_CAL = 1.98720425864083


def _kf(A, beta, Ea, T):
    T = np.asarray(T, dtype=np.longdouble)
    return np.longdouble(A) * T ** np.longdouble(beta) * np.exp(-np.longdouble(Ea) / (np.longdouble(R_CAL) * T))


def _conc(m, phi, par):
    """Concentrations of a CONP state written out: C_k = n_k / V, C_N2 by
    the ideal-gas law."""
    T, V, P = phi[0], phi[1], par
    C = phi[2:] / V
    return T, V, np.concatenate([C, (P / (R * T) - C.sum(axis=0))[None]], axis=0)


def _both(m, n=6, seed=3):
    phi, par = synth.make_states(m, n, seed, synth.CONP)
    Je = oracle.jacobian(m, synth.CONP, phi, par)
    Ja = oracle.jacobian(m, synth.CONP, phi, par, form=oracle.APPROX)
    return phi, par, Je, Ja


def test_bath_reactant_by_hand():
    """O + N2 -> NO + N (irreversible): q = kf C_O C_N2 with C_N2 = C_tot -
    sum C_k, so dq/dn_j = kf (delta_jO C_N2 - C_O) / V exactly and
    kf delta_jO C_N2 / V in the approximate form; row k is V nu_k dq/dn_j."""
    m = tm.single(dict(reac=[(O, 1), (N2, 1)], prod=[(NO, 1), (N, 1)], A=3.0e10, beta=0.4, Ea=9000.0, rev=False))
    phi, par, Je, Ja = _both(m)
    T, V, C = _conc(m, phi, par)
    kf = _kf(m.A[0], m.beta[0], m.Ea[0], T).astype(np.float64)
    nu = {O: -1.0, NO: 1.0, N: 1.0}
    for k, v in nu.items():
        for j in range(m.n_species - 1):
            exact = v * kf * ((j == O) * C[N2] - C[O])
            approx = v * kf * (j == O) * C[N2]
            np.testing.assert_allclose(Je[2 + k, 2 + j], exact, rtol=1e-11, atol=0)
            np.testing.assert_allclose(Ja[2 + k, 2 + j], approx, rtol=1e-11, atol=0)


def test_bath_efficiency_by_hand():
    """H + H + M -> H2 + M (irreversible) with alpha_N2 = 2, alpha_H2O = 3:
    [M] = sum alpha_k C_k, d[M]/dn_j = (alpha_j - alpha_N2) / V exactly and
    (alpha_j - 1) / V in the approximate form (bath gas at unit efficiency)."""
    m = tm.single(dict(reac=[(H, 2)], prod=[(H2, 1)], A=1.5e12, beta=-1.1, Ea=0.0, kind=synth.THIRD_BODY,
                       rev=False, eff={N2: 2.0, H2O: 3.0}))
    phi, par, Je, Ja = _both(m)
    T, V, C = _conc(m, phi, par)
    kf = _kf(m.A[0], m.beta[0], m.Ea[0], T).astype(np.float64)
    alpha = np.ones(m.n_species)
    alpha[N2], alpha[H2O] = 2.0, 3.0
    M = alpha @ C
    for k, v in ((H, -2.0), (H2, 1.0)):
        for j in range(m.n_species - 1):
            base = 2 * C[H] * (j == H) * M
            exact = v * kf * (base + C[H] ** 2 * (alpha[j] - alpha[N2]))
            approx = v * kf * (base + C[H] ** 2 * (alpha[j] - 1.0))
            np.testing.assert_allclose(Je[2 + k, 2 + j], exact, rtol=1e-11, atol=1e-300)
            np.testing.assert_allclose(Ja[2 + k, 2 + j], approx, rtol=1e-11, atol=1e-300)
    # only H and H2O columns survive in the approximate species rows
    cols = [j for j in range(m.n_species - 1) if np.any(Ja[2 + H, 2 + j] != 0)]
    assert sorted(cols) == sorted([H, H2O])


def test_no_bath_path_means_no_difference():
    """Without the bath gas in any rate and with unit bath-gas efficiencies,
    the two forms are the same function's derivative."""
    rx = [
        dict(reac=[(H, 1), (O2, 1)], prod=[(OH, 1), (O, 1)], A=2.0e11, beta=-0.3, Ea=15000.0),
        dict(reac=[(H, 1), (OH, 1)], prod=[(H2O, 1)], A=2.0e16, beta=-1.9, kind=synth.THIRD_BODY,
             eff={H2: 0.7, H2O: 3.5}),
        dict(reac=[(OH, 2)], prod=[(H2, 1), (O2, 1)], A=7.0e10, beta=-0.4, kind=synth.TROE,
             A0=2.0e12, beta0=-0.8, Ea0=-1500.0, troe=(0.7, 90.0, 1800.0, 5000.0), eff={H2O: 6.0}),
    ]
    m = synth.build_mechanism("no_bath", tm.SP, rx, seed=5)
    phi, par, Je, Ja = _both(m)
    np.testing.assert_allclose(Ja, Je, rtol=1e-12, atol=1e-300)
    assert np.array_equal(oracle.sparsity_pattern(m, oracle.APPROX), oracle.sparsity_pattern(m))


@pytest.mark.parametrize("name", ["all_kinds", "bath_efficiency"])
def test_dropped_part_is_the_same_in_every_species_column(name):
    """What the approximate form drops is d/dn_j through C_Ns (-1/V) and the
    (1 - alpha_Ns)/V part of d[M]/dn_j: the same for every species column j.
    The T and S columns are untouched."""
    m = getattr(tm, name)()
    phi, par, Je, Ja = _both(m)
    assert np.array_equal(Je[:, :2], Ja[:, :2])
    D = Je[:, 2:] - Ja[:, 2:]                                  # [N, Ns-1, n]
    scale = np.abs(Je).max(axis=(1,), keepdims=True) + 1e-300
    spread = np.abs(D - D[:, :1]) / scale
    assert spread.max() <= 1e-10, spread.max()
    assert np.abs(D).max() > 0                                  # something is dropped


@pytest.mark.parametrize("name", ["all_kinds", "bath_efficiency"])
def test_approx_pattern_superset_tight_and_subset_of_exact(name):
    m = getattr(tm, name)()
    pa = oracle.sparsity_pattern(m, oracle.APPROX)
    pe = oracle.sparsity_pattern(m)
    assert np.all(pe[pa])                                       # approx pattern within the exact one
    assert pa.sum() < pe.sum()
    phi, par = synth.make_states(m, 24, 17, synth.CONP)
    Ja = oracle.jacobian(m, synth.CONP, phi, par, form=oracle.APPROX)
    nz = np.any(Ja != 0, axis=2)
    assert not np.any(nz & ~pa)                                 # superset
    N = m.n_species + 1
    forced = np.zeros_like(pa)
    forced[:2, :] = forced[:, :2] = True
    forced[np.arange(N), np.arange(N)] = True
    assert np.all(nz[pa & ~forced])                             # tight


def test_workload_density_drops():
    """Sec. 3.4 reports the approximate form some 3-7 % less dense; the
    synthetic 53-species mechanism's bath gas (N2) sits in a few rates."""
    m = synth.make_mechanism("gri53")
    pa = oracle.sparsity_pattern(m, oracle.APPROX)
    pe = oracle.sparsity_pattern(m)
    N2_ = (m.n_species + 1) ** 2
    drop = (pe.sum() - pa.sum()) / N2_
    assert np.all(pe[pa]) and drop > 0.0
