"""Pins of the oracle's vector-Jacobian product (oracle.forms.vjp), the
differentiation form of the source terms of Sec. 2.2.

* The state part g_Phi = (dy/dPhi)^T u, y = (wdot_0 .. wdot_{Ns-1}, dT/dt),
  against the complex-step Jacobian of the source terms f (pinned by
  test_oracle_pins.py) through the identities that tie y to f:
    dwdot_k/dPhi_j = (J[k+2, j] - delta_{j,V} wdot_k) / V   (CONP, k < Ns-1)
    dwdot_k/dPhi_j = J[k+2, j] / V                          (CONV, k < Ns-1)
    dwdot_Ns/dPhi_j = -(1/W_Ns) sum_{k<Ns-1} W_k dwdot_k/dPhi_j
        (mass conservation of element-balanced reactions)
    d(dT/dt)/dPhi_j = J[0, j].
* The parameter part g_theta = sum_s (dy/dtheta)^T u, theta_i = (ln A_i,
  beta_i, Ea_i), against central differences of sum_s u . y over copies of
  one-reaction mechanisms (one of every kind) with that reaction's ln A, beta
  or Ea moved by +-delta (the mechanism data itself, not the oracle's
  parameter overrides).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import tiny_mechs as tm

U = 2.0 ** -53
H, O, H2, O2, OH, H2O, HO2, N, NO, N2 = range(10)


def _y_jacobian_from_f(m, mode, phi, par):
    """dy/dPhi [Ns+1, N, n] and an absolute rounding envelope of it, both from
    the Jacobian of f and its envelope."""
    J, env = oracle.jacobian_envelope(m, mode, phi, par)
    f = oracle.source_terms(m, mode, phi, par)
    ns, n = m.n_species, phi.shape[1]
    V = phi[1] if mode == synth.CONP else par
    Jy = np.zeros((ns + 1, ns + 1, n))
    Ey = np.zeros_like(Jy)
    for k in range(ns - 1):
        Jy[k] = J[k + 2] / V
        Ey[k] = env[k + 2] / V
        if mode == synth.CONP:
            wk = f[k + 2] / V
            Jy[k, 1] = (J[k + 2, 1] - wk) / V
            Ey[k, 1] += np.abs(wk) / V
    ratio = m.W[:-1] / m.W[-1]
    Jy[ns - 1] = -np.einsum("k,kjn->jn", ratio, Jy[: ns - 1])
    Ey[ns - 1] = np.einsum("k,kjn->jn", ratio, Ey[: ns - 1])
    Jy[ns] = J[0]
    Ey[ns] = env[0]
    return Jy, Ey


@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
@pytest.mark.parametrize("name", ["all_kinds", "bath_efficiency", "all_types", "h2co13"])
def test_vjp_state_part_equals_u_times_jacobian_identities(mechs, name, mode):
    m = getattr(tm, name)() if name in ("all_kinds", "bath_efficiency", "all_types") else mechs(name)
    n = 5
    phi, par = synth.make_states(m, n, 31 + mode, mode)
    uw, uT = synth.make_cotangents(m.n_species, n, 31)
    g_phi, _ = oracle.vjp(m, mode, phi, par, uw, uT)
    Jy, Ey = _y_jacobian_from_f(m, mode, phi, par)
    u = np.concatenate([uw, uT[None]], axis=0)
    want = np.einsum("rn,rjn->jn", u, Jy)
    env = np.einsum("rn,rjn->jn", np.abs(u), np.maximum(Ey, np.abs(Jy)))
    err = np.abs(g_phi - want)
    assert np.all(err <= 1e-10 * env + 1e-300), float(np.max(err / (env + 1e-300)))


def _one_reaction_cases():
    """One reaction of every kind (inputs only; arbitrary parameters)."""
    return [
        ("elementary", dict(reac=[(H, 1), (O2, 1)], prod=[(OH, 1), (O, 1)], A=2.0e11, beta=-0.3, Ea=15000.0)),
        ("irreversible", dict(reac=[(O, 1), (H2, 1)], prod=[(OH, 1), (H, 1)], A=4.0e4, beta=2.5, Ea=6000.0,
                              rev=False)),
        ("second order", dict(reac=[(OH, 2)], prod=[(O, 1), (H2O, 1)], A=3.0e1, beta=3.0, Ea=-1500.0)),
        ("third body", dict(reac=[(H, 1), (OH, 1)], prod=[(H2O, 1)], A=2.0e16, beta=-1.9, Ea=300.0,
                            kind=synth.THIRD_BODY, eff={H2: 0.7, H2O: 3.5})),
        ("lindemann", dict(reac=[(H, 1), (O2, 1)], prod=[(HO2, 1)], A=5.0e9, beta=0.4, Ea=800.0,
                           kind=synth.LINDEMANN, A0=6.0e14, beta0=-1.7, Ea0=500.0, eff={H2: 2.0, H2O: 12.0})),
        ("troe 4", dict(reac=[(OH, 2)], prod=[(H2, 1), (O2, 1)], A=7.0e10, beta=-0.4, Ea=1200.0, kind=synth.TROE,
                        A0=2.0e12, beta0=-0.8, Ea0=-1500.0, troe=(0.7, 90.0, 1800.0, 5000.0), eff={H2O: 6.0})),
        ("troe 3", dict(reac=[(HO2, 1)], prod=[(H, 1), (O2, 1)], A=5.0e14, beta=0.0, Ea=40000.0, kind=synth.TROE,
                        A0=1.0e16, beta0=-1.0, Ea0=30000.0, troe=(0.5, 100.0, 2000.0), eff={H2: 1.5})),
        ("sri", dict(reac=[(H, 1), (HO2, 1)], prod=[(H2, 1), (O2, 1)], A=2.0e10, beta=0.3, Ea=2000.0,
                     kind=synth.SRI, A0=3.0e14, beta0=-1.5, Ea0=1000.0, sri=(0.45, 800.0, 1000.0, 1.1, -0.2),
                     eff={O2: 0.4})),
        ("chemically activated", dict(reac=[(H, 1), (O2, 1)], prod=[(HO2, 1)], A=5.0e9, beta=0.4, Ea=700.0,
                                      kind=synth.LINDEMANN, chem=True, A0=6.0e14, beta0=-1.7, Ea0=500.0,
                                      eff={H2: 2.0})),
        ("explicit reverse", dict(reac=[(H, 1), (O2, 1)], prod=[(OH, 1), (O, 1)], A=2.0e11, beta=-0.3,
                                  Ea=15000.0, rev_arr=(1.5e10, 0.1, 800.0))),
        ("bath gas reactant", dict(reac=[(N, 1), (NO, 1)], prod=[(N2, 1), (O, 1)], A=3.0e10, beta=0.2,
                                   Ea=400.0)),
    ]


def _perturbed(m, p, sign):
    """Copy of one-reaction mechanism m with theta_p moved by sign * delta_p;
    returns (copy, delta_p)."""
    c = m.copy()
    if p == 0:                       # ln A
        d = 1e-5
        c.A[0] = m.A[0] * math.exp(sign * d)
    elif p == 1:                     # beta
        d = 1e-6
        c.beta[0] = m.beta[0] + sign * d
    else:                            # Ea [cal/mol]
        d = 1e-6 * max(abs(m.Ea[0]), 100.0)
        c.Ea[0] = m.Ea[0] + sign * d
    return c, d


@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
@pytest.mark.parametrize("label,rx", _one_reaction_cases(), ids=[c[0] for c in _one_reaction_cases()])
def test_vjp_parameter_part_equals_central_differences(label, rx, mode):
    m = tm.single(rx)
    n = 4
    phi, par = synth.make_states(m, n, 57 + mode, mode)
    uw, uT = synth.make_cotangents(m.n_species, n, 57)
    _, g_theta = oracle.vjp(m, mode, phi, par, uw, uT)
    u = np.concatenate([uw, uT[None]], axis=0)
    for p in range(3):
        mp, d = _perturbed(m, p, +1)
        mm, _ = _perturbed(m, p, -1)
        dy = (oracle.outputs_y(mp, mode, phi, par) - oracle.outputs_y(mm, mode, phi, par)) / (2 * d)
        per_state = np.sum(u * dy, axis=0)
        fd = per_state.sum()
        scale = np.sum(np.abs(u * dy)) + 1e-300
        assert abs(g_theta[0, p] - fd) <= 1e-6 * scale, (label, p, g_theta[0, p], fd, scale)


@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
def test_vjp_parameter_part_on_a_whole_mechanism(mode):
    """On a whole mechanism (every kind): g_theta[i] against central
    differences of sum_s u . y with reaction i's parameter moved, the
    tolerance widened by the rounding of y itself (the other reactions'
    terms)."""
    m = tm.all_kinds()
    n = 6
    phi, par = synth.make_states(m, n, 91 + mode, mode)
    uw, uT = synth.make_cotangents(m.n_species, n, 91)
    _, g = oracle.vjp(m, mode, phi, par, uw, uT)
    u = np.concatenate([uw, uT[None]], axis=0)
    tight = 0
    for i in range(m.n_reactions):
        for p in range(3):
            d = (1e-5, 1e-6, 1e-6 * max(abs(m.Ea[i]), 100.0))[p]
            mp, mm = m.copy(), m.copy()
            if p == 0:
                mp.A[i], mm.A[i] = m.A[i] * math.exp(d), m.A[i] * math.exp(-d)
            elif p == 1:
                mp.beta[i], mm.beta[i] = m.beta[i] + d, m.beta[i] - d
            else:
                mp.Ea[i], mm.Ea[i] = m.Ea[i] + d, m.Ea[i] - d
            yp, ym = oracle.outputs_y(mp, mode, phi, par), oracle.outputs_y(mm, mode, phi, par)
            fd = np.sum(u * (yp - ym)) / (2 * d)
            rounding = 64 * U * np.sum(np.abs(u) * (np.abs(yp) + np.abs(ym))) / (2 * d)
            assert abs(g[i, p] - fd) <= 1e-5 * abs(fd) + rounding, (i, p, g[i, p], fd, rounding)
            tight += rounding < 1e-3 * abs(fd)
    assert tight >= m.n_reactions * 3 // 2      # most checks are far tighter than O(1)
