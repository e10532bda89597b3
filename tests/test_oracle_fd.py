"""Pin of the oracle's first-order forward finite-difference Jacobian (the
comparator of Sec. 3.5.2) against the complex-step Jacobian: a forward
difference with step h_j is off by its truncation error (here within 1e-6
of the Jacobian's rounding envelope: h_j is about 1.5e-8 |Phi_j|) plus the
rounding of the two source-term evaluations divided by h_j."""
import numpy as np
import pytest

import oracle
import synth
from tests import tiny_mechs as tm

U = 2.0 ** -53


def _mech(name):
    return getattr(tm, name)() if name in ("all_kinds", "bath_efficiency", "all_types") else synth.make_mechanism(name)


def fd_tolerance(m, mode, phi, par):
    _, env = oracle.jacobian_envelope(m, mode, phi, par)
    _, envf = oracle.source_term_envelope(m, mode, phi, par)
    h = oracle.fd_steps(m, mode, phi, par)
    return 1e-6 * env + 64 * U * envf[:, None, :] / h[None, :, :]


@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
@pytest.mark.parametrize("name", ["all_kinds", "bath_efficiency", "all_types", "h2co13", "gri53"])
def test_fd_jacobian_within_truncation_and_rounding(name, mode):
    m = _mech(name)
    phi, par = synth.make_states(m, 12, 31, mode)
    Jf, f0 = oracle.fd_jacobian(m, mode, phi, par)
    J = oracle.jacobian(m, mode, phi, par)
    assert np.array_equal(f0, oracle.source_terms(m, mode, phi, par))
    tol = fd_tolerance(m, mode, phi, par)
    assert np.all(np.abs(Jf - J) <= tol), float(np.max(np.abs(Jf - J) / tol))
    # the bound has teeth: the same differences assigned to the neighbouring
    # column, or taken backwards, fail it
    assert not np.all(np.abs(np.roll(Jf, 1, axis=1) - J) <= tol)
    assert not np.all(np.abs(-Jf - J) <= tol)


def test_fd_steps_are_exact_scalings():
    m = _mech("gri53")
    phi, par = synth.make_states(m, 50, 2, synth.CONP)
    h = oracle.fd_steps(m, synth.CONP, phi, par)
    assert np.all(h > 0)
    rel = h / np.abs(phi)
    big = np.abs(phi) > 2.0 ** -26 * (phi[1] * par / (oracle.R * phi[0]))[None, :]
    # realised step = 2^-26 |Phi_j| up to the rounding of Phi_j + delta_j
    assert np.all(np.abs(rel[big] / 2.0 ** -26 - 1.0) <= 2.0 ** -25)
