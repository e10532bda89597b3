"""CPU oracle for the derived forms: Newton iteration matrix and the
vector-Jacobian product of the production rates and dT/dt.

TEST INFRASTRUCTURE ONLY (same rules as ``oracle.kinetics``).

* Newton matrix M = I - h gamma J (the matrix an implicit integrator factors;
  the paper motivates the Jacobian by implicit integration, Sec. 1 and
  Sec. 3.4), here in float64.
* VJP of y = (wdot_0 .. wdot_{Ns-1}, dT/dt): g_Phi = (dy/dPhi)^T u per state
  and g_theta = sum over states of (dy/dtheta)^T u for the per-reaction
  parameters theta_i = (ln A_i, beta_i, Ea_i) of the high-pressure (or only)
  Arrhenius set, all by complex-step differentiation.
* First-order forward finite-difference Jacobian, the comparator of
  Sec. 3.5.2 (the analytical Jacobian's speedup over it): column j is
  (f(Phi + h_j e_j) - f(Phi)) / h_j.  The paper gives no step rule; this one
  uses delta_j = 2^-26 max(|Phi_j|, 2^-26 n_tot), n_tot = P V / (R T), and
  the realised step h_j = (Phi_j + delta_j) - Phi_j.
"""
from __future__ import annotations

import numpy as np

from .kinetics import CONP, R, rates, source_terms, source_terms_from_rates, jacobian, _cs_step


def newton_matrix(mech, mode, phi, param, h, gamma=1.0):
    """Dense I - h gamma J, shape [N, N, n]."""
    J = jacobian(mech, mode, phi, param)
    N = J.shape[0]
    M = -(h * gamma)[None, None, :] * J if np.ndim(h) else -(h * gamma) * J
    M[np.arange(N), np.arange(N)] += 1.0
    return M


def outputs_y(mech, mode, phi, param, **over):
    """y = (wdot_0 .. wdot_{Ns-1}, dT/dt), shape [Ns+1, n]."""
    r = rates(mech, mode, phi, param, **over)
    f, _ = source_terms_from_rates(mech, mode, r)
    return np.concatenate([r["wdot"], f[:1]], axis=0)


def y_jacobian(mech, mode, phi, param):
    """dy/dPhi [Ns+1, Ns+1, n] by complex-step differentiation."""
    N = mech.n_species + 1
    Jy = np.empty((N, N, phi.shape[1]))
    for j in range(N):
        ph = phi.astype(np.complex128)
        hj = _cs_step(phi[j])
        ph[j] = ph[j] + 1j * hj
        Jy[:, j] = outputs_y(mech, mode, ph, param.astype(np.complex128)).imag / hj
    return Jy


def vjp_envelope(mech, mode, phi, param, u_wdot, u_T):
    """Absolute envelopes of the VJP: sum of |u_y dy/dPhi_j| per state, and
    sum over states of |w_q dq_i/dtheta| per reaction parameter."""
    Jy = y_jacobian(mech, mode, phi, param)
    u = np.concatenate([u_wdot, u_T[None, :]], axis=0)
    env_phi = np.sum(np.abs(u)[:, None, :] * np.abs(Jy), axis=0)
    return env_phi, _theta_terms(mech, mode, phi, param, u_wdot, u_T, absolute=True)


def _theta_terms(mech, mode, phi, param, u_wdot, u_T, absolute=False):
    r0 = rates(mech, mode, phi, param)
    _, aux = source_terms_from_rates(mech, mode, r0)
    nu = r0["nu"].astype(float)                                 # [Ns, Nr]
    # dy/dq_i per state: wdot_k -> nu_ki ; dT/dt -> -sum_k E_k nu_ki / den
    E = aux["E"]                                                # [Ns, n]
    w_q = (nu.T @ u_wdot)                                        # [Nr, n]
    w_q = w_q - (nu.T @ E) * (u_T / aux["den"])[None, :]
    f = np.abs if absolute else (lambda x: x)
    g_theta = np.zeros((mech.n_reactions, 3))
    hA = 1e-30
    A_c = mech.A * np.exp(1j * hA)
    q = rates(mech, mode, phi.astype(np.complex128), param.astype(np.complex128), A=A_c)["q"]
    g_theta[:, 0] = np.sum(f(w_q * (q.imag / hA)), axis=1)
    hb = 1e-30
    q = rates(mech, mode, phi.astype(np.complex128), param.astype(np.complex128),
              beta=mech.beta + 1j * hb)["q"]
    g_theta[:, 1] = np.sum(f(w_q * (q.imag / hb)), axis=1)
    hE = _cs_step(mech.Ea)
    q = rates(mech, mode, phi.astype(np.complex128), param.astype(np.complex128),
              Ea=mech.Ea + 1j * hE)["q"]
    g_theta[:, 2] = np.sum(f(w_q * (q.imag / hE[:, None])), axis=1)
    return g_theta


def vjp(mech, mode, phi, param, u_wdot, u_T):
    """(g_phi [Ns+1, n], g_theta [Nr, 3]) with g_theta summed over states."""
    ns, N = mech.n_species, mech.n_species + 1
    u = np.concatenate([u_wdot, u_T[None, :]], axis=0)        # [Ns+1, n]
    g_phi = np.empty_like(phi)
    for j in range(N):
        ph = phi.astype(np.complex128)
        hj = _cs_step(phi[j])
        ph[j] = ph[j] + 1j * hj
        y = outputs_y(mech, mode, ph, param.astype(np.complex128))
        g_phi[j] = np.sum(u * (y.imag / hj), axis=0)
    # parameter derivatives: q_i depends only on reaction i's own parameters,
    # so one complex evaluation per parameter kind gives d q_i / d theta_i for
    # every i at once; y is then linear in q.
    return g_phi, _theta_terms(mech, mode, phi, param, u_wdot, u_T)


FD_SCALE = 2.0 ** -26        # about sqrt(unit roundoff); a power of two, so scaling is exact


def fd_steps(mech, mode, phi, param):
    """Realised forward-difference steps h [N, n] of fd_jacobian."""
    T = phi[0]
    V, P = (phi[1], param) if mode == CONP else (param, phi[1])
    ntot = (P * V) / (R * T)
    h = np.empty_like(phi)
    for j in range(phi.shape[0]):
        d = FD_SCALE * np.maximum(np.abs(phi[j]), FD_SCALE * ntot)
        h[j] = (phi[j] + d) - phi[j]
    return h


def fd_jacobian(mech, mode, phi, param):
    """Dense first-order forward finite-difference Jacobian [N, N, n] and the
    source terms at Phi (Sec. 3.5.2's comparator; step rule in the module
    notes)."""
    N = phi.shape[0]
    f0 = source_terms(mech, mode, phi, param)
    h = fd_steps(mech, mode, phi, param)
    J = np.empty((N, N, phi.shape[1]))
    for j in range(N):
        x = phi.copy()
        x[j] = phi[j] + h[j]
        J[:, j] = (source_terms(mech, mode, x, param) - f0) / h[j]
    return J, f0
