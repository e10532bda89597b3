"""GPU parity of the approximate Jacobian form (Sec. 3.4, "Sparsity
patterns") against the oracle's approximate form, through the C ABI."""
import numpy as np
import pytest

import oracle
import synth
from tests import tiny_mechs as tm
from tests.parity import RTOL_JAC, ATOL_JAC, RTOL_SRC, ATOL_SRC, check_close, newton_tol, jacobian_layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pj():
    import paper_1809_01029_gb300 as pj
    from paper_1809_01029_gb300 import build
    build.build()
    pj.load_library()
    return pj


def _mech(mechs, name):
    if name in ("all_kinds", "bath_efficiency", "all_types"):
        return getattr(tm, name)()
    return mechs(name)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [("all_kinds", 40), ("bath_efficiency", 35), ("all_types", 31), ("h2co13", 100), ("gri53", 64), ("gri53_types", 40), ("usc111", 16)]


@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
@pytest.mark.parametrize("name,n", CASES)
def test_approximate_jacobian_matches_oracle(pj, mechs, name, n, mode):
    """Every format against the oracle's approximate form; the envelope of
    the exact form bounds the rounding (the approximate form drops terms).
    The source terms computed on the way are those of the exact handle."""
    import torch
    m = _mech(mechs, name)
    h = pj.pj_mech_create(m)
    ha = h.with_jacobian_form(pj.PJ_JAC_APPROX)
    phi, par = synth.make_states(m, n, 900 + n, mode)
    Ja = oracle.jacobian(m, mode, phi, par, form=oracle.APPROX)
    _, env = oracle.jacobian_envelope(m, mode, phi, par)
    d_phi, d_par = dev(phi), dev(par)
    N1 = m.n_species + 1
    f_a = torch.empty((N1, n), dtype=torch.float64, device="cuda")
    f_e = torch.empty((N1, n), dtype=torch.float64, device="cuda")
    Jd = pj.jacobian_dense(ha, mode, d_phi, d_par, dphi=f_a).cpu().numpy().reshape(N1, N1, n)
    check_close(Jd, Ja, env, RTOL_JAC, ATOL_JAC, f"{name} approx dense mode={mode}")
    mask = oracle.sparsity_pattern(m, oracle.APPROX)
    assert np.all(Jd[~mask] == 0.0)
    pj.jacobian_dense(h, mode, d_phi, d_par, dphi=f_e)
    f_ref, f_env = oracle.source_term_envelope(m, mode, phi, par)
    check_close(f_a.cpu().numpy(), f_ref, f_env, RTOL_SRC, ATOL_SRC, f"{name} f of the approximate form")
    check_close(f_e.cpu().numpy(), f_ref, f_env, RTOL_SRC, ATOL_SRC, f"{name} f of the exact form")
    for fmt, conv in ((pj.PJ_CSR, oracle.dense_to_csr_values), (pj.PJ_CSC, oracle.dense_to_csc_values)):
        vals = pj.jacobian_sparse(ha, mode, d_phi, d_par, fmt=fmt).cpu().numpy()
        assert vals.shape[0] == ha.nnz
        check_close(vals, conv(m, Ja, oracle.APPROX), conv(m, env, oracle.APPROX), RTOL_JAC, ATOL_JAC,
                    f"{name} approx fmt={fmt} mode={mode}")


def test_approximate_newton_matrix(pj, mechs):
    """FP32 M = I - h gamma J on the approximate pattern, at the accuracy
    stated for the FP32 form (tests/parity.py: newton_tol)."""
    m = mechs("gri53")
    ha = pj.pj_mech_create(m).with_jacobian_form(pj.PJ_JAC_APPROX)
    n = 40
    phi, par = synth.make_states(m, n, 41, synth.CONP)
    hs = synth.make_step_sizes(n, 41)
    Ja = oracle.jacobian(m, synth.CONP, phi, par, form=oracle.APPROX)
    _, env = oracle.jacobian_envelope(m, synth.CONP, phi, par)
    N1 = m.n_species + 1
    M_ref = -hs[None, None, :] * Ja
    M_ref[np.arange(N1), np.arange(N1)] += 1.0
    scale = np.abs(M_ref) + hs[None, None, :] * env
    Ms = pj.newton_matrix_f32(ha, synth.CONP, dev(phi), dev(par), dev(hs), 1.0, fmt=pj.PJ_CSR)
    Ms = Ms.cpu().numpy().astype(np.float64)
    e = np.abs(Ms - oracle.dense_to_csr_values(m, M_ref, oracle.APPROX))
    assert np.all(e <= newton_tol(oracle.dense_to_csr_values(m, scale, oracle.APPROX)))


def test_approximate_form_through_a_plan(pj, mechs):
    """Uneven batches through a persistent-kernel plan on the approximate
    handle give the values of the direct entry point."""
    import torch
    m = mechs("gri53")
    ha = pj.pj_mech_create(m).with_jacobian_form(pj.PJ_JAC_APPROX)
    sizes = [37, 300, 5]
    batches, ref = [], []
    for b, n in enumerate(sizes):
        phi, par = synth.make_states(m, n, 60 + b, synth.CONP)
        d_phi, d_par = dev(phi), dev(par)
        out = torch.empty((ha.nnz, n), dtype=torch.float64, device="cuda")
        f = torch.empty((m.n_species + 1, n), dtype=torch.float64, device="cuda")
        batches.append((d_par, d_phi, out, f))
        with jacobian_layout("percore"):  # the plan's one-state-per-thread arithmetic
            ref.append(pj.jacobian_sparse(ha, synth.CONP, d_phi, d_par).cpu().numpy())
    plan = pj.Plan(ha, pj.PJ_OP_JACOBIAN, synth.CONP, batches)
    plan.run()
    torch.cuda.synchronize()
    for (_, _, out, _), r in zip(batches, ref):
        np.testing.assert_allclose(out.cpu().numpy(), r, rtol=1e-12, atol=1e-300)
