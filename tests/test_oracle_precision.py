"""Extended-precision reference for the FP64 oracle.

The same oracle code evaluated in np.longdouble (x87 extended on x86-64: a
64-bit significand, eps 1.1e-19; IEEE quad on AArch64) bounds the FP64
oracle's own rounding error: source terms and the complex-step Jacobian
(Sec. 2.2) of sampled states agree with the extended evaluation within a
small multiple of u = 2^-53 times the oracle's rounding envelope, far inside
the parity tolerances (1e-10 and 1e-8 times the envelope), so the oracle's
own rounding cannot decide a GPU parity verdict.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import tiny_mechs as tm
from tests.parity import RTOL_JAC, RTOL_SRC

U = 2.0 ** -53
K_SRC = 2048.0      # observed at most ~500 on these workloads
K_JAC = 8192.0      # observed at most ~1300


def _mech(mechs, name):
    return getattr(tm, name)() if name in ("all_kinds", "all_types") else mechs(name)


@pytest.mark.skipif(np.finfo(np.longdouble).eps > 2.0 ** -60, reason="no extended long double on this host")
@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
@pytest.mark.parametrize("name,n", [("all_kinds", 6), ("all_types", 6), ("h2co13", 8), ("gri53", 3)])
def test_fp64_oracle_within_its_envelope_of_the_extended_evaluation(mechs, name, n, mode):
    m = _mech(mechs, name)
    phi, par = synth.make_states(m, n, 808 + n, mode)
    phl, pal = phi.astype(np.longdouble), par.astype(np.longdouble)
    f64, fenv = oracle.source_term_envelope(m, mode, phi, par)
    fl = oracle.source_terms(m, mode, phl, pal)
    assert fl.dtype == np.longdouble
    err = np.abs(f64 - fl)
    assert np.all(err <= K_SRC * U * fenv), float(np.max(err / (U * np.maximum(fenv, 1e-300))))
    J, env = oracle.jacobian_envelope(m, mode, phi, par)
    Jl = oracle.jacobian(m, mode, phl, pal)
    assert Jl.dtype == np.longdouble
    err = np.abs(J - Jl)
    assert np.all(err <= K_JAC * U * env), float(np.max(err / (U * np.maximum(env, 1e-300))))
    # the parity tolerances are far above the oracle's own rounding
    assert RTOL_JAC >= 1000 * K_JAC * U and RTOL_SRC >= 100 * K_SRC * U
