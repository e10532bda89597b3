"""GPU parity of the finite-difference Jacobian comparator (Sec. 3.5.2).

The steps are exact power-of-two scalings, so the kernel and the oracle
perturb identical bits.  (1) Bit for bit, every column equals the GPU
source-term kernel at the perturbed states minus that at Phi, over h_j.
(2) Against the oracle's finite differences the only difference is the
rounding of the source terms divided by h_j; source terms of the two sides
agree to about 1000 u env where one exp dominates (exp(x) carries a relative
rounding of about |x| u from its rounded argument, |x| up to ~100 here, and
the sides form the arguments differently), so the bound is 2 * 4096 u
env_f / h_j.  (3) Against the exact Jacobian, the oracle pin's truncation
and rounding bound plus (2)'s."""
import numpy as np
import pytest

import oracle
import synth
from tests import tiny_mechs as tm
from tests.test_oracle_fd import fd_tolerance

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module")
def pj():
    import paper_1809_01029_gb300 as pj
    from paper_1809_01029_gb300 import build
    build.build()
    pj.load_library()
    return pj


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _mech(mechs, name):
    return getattr(tm, name)() if name in ("all_kinds", "bath_efficiency", "all_types") else mechs(name)


@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
@pytest.mark.parametrize("name,n", [("all_kinds", 37), ("bath_efficiency", 20), ("all_types", 25), ("h2co13", 130), ("gri53", 33), ("gri53_types", 21)])
def test_fd_jacobian_matches_oracle(pj, mechs, name, n, mode):
    import torch
    m = _mech(mechs, name)
    h = pj.pj_mech_create(m)
    phi, par = synth.make_states(m, n, 500 + n, mode)
    Jf, f0 = oracle.fd_jacobian(m, mode, phi, par)
    _, envf = oracle.source_term_envelope(m, mode, phi, par)
    hs = oracle.fd_steps(m, mode, phi, par)
    tol = 2 * 4096 * U * envf[:, None, :] / hs[None, :, :]
    N1 = m.n_species + 1
    d_phi, d_par = dev(phi), dev(par)
    f = torch.empty((N1, n), dtype=torch.float64, device="cuda")
    Jd = pj.jacobian_fd(h, mode, d_phi, d_par, fmt=pj.PJ_DENSE, dphi=f).cpu().numpy().reshape(N1, N1, n)
    # (1) the kernel's differences are those of the source-term kernel
    f0 = pj.source_terms(h, mode, d_phi, d_par).cpu().numpy()
    assert np.array_equal(f.cpu().numpy(), f0)
    for j in range(N1):
        x = phi.copy()
        x[j] = phi[j] + hs[j]
        f1 = pj.source_terms(h, mode, dev(x), d_par).cpu().numpy()
        assert np.array_equal(Jd[:, j], (f1 - f0) / hs[j]), j
    # (2) the oracle's finite differences
    err = np.abs(Jd - Jf)
    bad = err > tol
    assert not bad.any(), (np.argwhere(bad)[:3], float(np.max(err[bad] / tol[bad])))
    # (3) the exact Jacobian
    J = oracle.jacobian(m, mode, phi, par)
    assert np.all(np.abs(Jd - J) <= fd_tolerance(m, mode, phi, par) + tol)
    for fmt, conv in ((pj.PJ_CSR, oracle.dense_to_csr_values), (pj.PJ_CSC, oracle.dense_to_csc_values)):
        vals = pj.jacobian_fd(h, mode, d_phi, d_par, fmt=fmt).cpu().numpy()
        assert np.array_equal(vals, conv(m, Jd)), fmt          # same kernel arithmetic, other storage


def test_fd_invalid_state_is_nan_and_counted(pj, mechs):
    import torch
    m = mechs("h2co13")
    h = pj.pj_mech_create(m)
    n = 40
    phi, par = synth.make_states(m, n, 8, synth.CONP)
    phi[0, 5] = -1.0
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    vals = pj.jacobian_fd(h, synth.CONP, dev(phi), dev(par), status=status).cpu().numpy()
    assert int(status.item()) == 1
    assert np.all(np.isnan(vals[:, 5]))
    assert np.all(np.isfinite(np.delete(vals, 5, axis=1)))
