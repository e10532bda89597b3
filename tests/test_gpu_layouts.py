"""GPU parity of the two Jacobian kernel families against the CPU oracle.

"coop": the warps of a block share a tile of 32 states (lane = state) and
split the reactions, species and columns among themselves; "percore": one
state per thread (shared memory, TMEM or a global workspace).  The library
picks the layout measured fastest; these tests force
each family on every mechanism so that both are checked everywhere, on
batches that span several tiles with a ragged tail, a padded leading
dimension, invalid states inside a tile and more tiles than one round of the
persistent grid.  Through the C ABI (the binding only marshals arguments).
"""
import numpy as np
import pytest

import oracle
import synth
from tests import tiny_mechs as tm
from tests.parity import (RTOL_SRC, ATOL_SRC, RTOL_JAC, ATOL_JAC, check_close, jacobian_layout, newton_tol,
                          newton_error)

pytestmark = pytest.mark.gpu

LAYOUTS = ["coop", "coop-global", "percore"]


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


def to_dev(a, ld=None):
    import torch
    a = np.asarray(a, dtype=np.float64)
    if ld is None or a.ndim == 1:
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    buf = torch.full((a.shape[0], ld), float("nan"), dtype=torch.float64, device="cuda")
    buf[:, : a.shape[1]] = torch.from_numpy(a).cuda()
    return buf[:, : a.shape[1]]


CASES = [("all_kinds", 45), ("bath_efficiency", 33), ("all_types", 70), ("h2co13", 97), ("gri53", 70),
         ("gri53_types", 39), ("usc111", 33)]


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
@pytest.mark.parametrize("name,n", CASES)
def test_layout_all_formats_match_oracle(pj, mechs, name, n, mode, layout):
    """Dense, CSR and CSC values and the source terms of each family against
    the oracle (tolerance of Sec. 3.2's cancellation reading: rtol times the
    larger of |J| and the oracle's envelope)."""
    import torch
    m = _mech(mechs, name)
    h = pj.pj_mech_create(m)
    phi, par = synth.make_states(m, n, 1300 + n, mode)
    J, env = oracle.jacobian_envelope(m, mode, phi, par)
    f_ref, f_env = oracle.source_term_envelope(m, mode, phi, par)
    N1 = m.n_species + 1
    d_phi, d_par = to_dev(phi, ld=n + 5), to_dev(par)
    # outputs share the states' leading dimension
    dphi = torch.full((N1, n + 5), float("nan"), dtype=torch.float64, device="cuda")[:, :n]
    with jacobian_layout(layout):
        Jd = pj.jacobian_dense(h, mode, d_phi, d_par, dphi=dphi).cpu().numpy().reshape(N1, N1, n)
        sparse = {fmt: pj.jacobian_sparse(h, mode, d_phi, d_par, fmt=fmt).cpu().numpy()
                  for fmt in (pj.PJ_CSR, pj.PJ_CSC)}
    check_close(Jd, J, env, RTOL_JAC, ATOL_JAC, f"{name} {layout} dense mode={mode}")
    assert np.all(Jd[~oracle.sparsity_pattern(m)] == 0.0)
    check_close(dphi.cpu().numpy(), f_ref, f_env, RTOL_SRC, ATOL_SRC, f"{name} {layout} source terms")
    for fmt, conv in ((pj.PJ_CSR, oracle.dense_to_csr_values), (pj.PJ_CSC, oracle.dense_to_csc_values)):
        check_close(sparse[fmt], conv(m, J), conv(m, env), RTOL_JAC, ATOL_JAC, f"{name} {layout} fmt={fmt}")


@pytest.mark.parametrize("layout", LAYOUTS)
def test_layout_invalid_states_inside_a_tile(pj, mechs, layout):
    """Invalid states (T <= 0, non-finite amounts, a bath-gas concentration
    below -1e-12 C_tot) get NaN outputs and are counted; their neighbours in
    the same 32-state tile are unaffected."""
    import torch
    m = mechs("gri53")
    h = pj.pj_mech_create(m)
    n = 100
    phi, par = synth.make_states(m, n, 77, synth.CONP)
    bad = [3, 40, 41, 99]
    phi[0, 3] = -5.0
    phi[7, 40] = np.nan
    phi[2:-1, 41] *= 10.0          # amounts far above P V / (R T): C_Ns < 0
    phi[1, 99] = np.inf
    good = np.setdiff1d(np.arange(n), bad)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    dphi = torch.empty((m.n_species + 1, n), dtype=torch.float64, device="cuda")
    with jacobian_layout(layout):
        vals = pj.jacobian_sparse(h, synth.CONP, to_dev(phi), to_dev(par), dphi=dphi, status=status)
    vals, dphi = vals.cpu().numpy(), dphi.cpu().numpy()
    assert int(status.item()) == len(bad)
    assert np.isnan(vals[:, bad]).all() and np.isnan(dphi[:, bad]).all()
    J, env = oracle.jacobian_envelope(m, synth.CONP, phi[:, good], par[good])
    check_close(vals[:, good], oracle.dense_to_csr_values(m, J), oracle.dense_to_csr_values(m, env), RTOL_JAC,
                ATOL_JAC, f"{layout} valid neighbours")


def test_coop_many_rounds_of_the_persistent_grid(pj, mechs):
    """More tiles than one round of the persistent grid (152 SMs x 32 states)
    with a ragged last tile: every state of the cooperative kernel within the
    oracle's tolerance on a sample spread over the rounds, and the whole
    batch within rounding of the sums of the one-state-per-thread layout."""
    m = mechs("h2co13")
    h = pj.pj_mech_create(m)
    n = 3 * 152 * 32 + 17
    phi, par = synth.make_states(m, n, 88, synth.CONV)
    d_phi, d_par = to_dev(phi), to_dev(par)
    with jacobian_layout("coop"):
        co = pj.jacobian_sparse(h, synth.CONV, d_phi, d_par).cpu().numpy()
    with jacobian_layout("percore"):
        pc = pj.jacobian_sparse(h, synth.CONV, d_phi, d_par).cpu().numpy()
    pick = np.concatenate([np.arange(0, n, 97), [n - 17, n - 1]])
    J, env = oracle.jacobian_envelope(m, synth.CONV, phi[:, pick], par[pick])
    ref, env = oracle.dense_to_csr_values(m, J), oracle.dense_to_csr_values(m, env)
    check_close(co[:, pick], ref, env, RTOL_JAC, ATOL_JAC, "coop sample")
    # two orders of the same sums: far inside the envelope tolerance
    scale = np.maximum(np.abs(pc), np.abs(co)).max(axis=0, keepdims=True)
    assert np.all(np.abs(co - pc) <= 1e-12 * scale)


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("name,n", [("gri53", 66), ("usc111", 35)])
def test_layout_newton_matrix_f32(pj, mechs, name, n, layout):
    """The FP32 Newton matrix of each family within the precision form's
    stated accuracy of the FP64 oracle (tests/parity.py: newton_tol)."""
    m = mechs(name)
    h = pj.pj_mech_create(m)
    phi, par = synth.make_states(m, n, 1900 + n, synth.CONP)
    hs = synth.make_step_sizes(n, 1900 + n)
    J, env = oracle.jacobian_envelope(m, synth.CONP, phi, par)
    N1 = m.n_species + 1
    M_ref = -hs[None, None, :] * J
    M_ref[np.arange(N1), np.arange(N1)] += 1.0
    scale = np.abs(M_ref) + hs[None, None, :] * env
    with jacobian_layout(layout):
        M = pj.newton_matrix_f32(h, synth.CONP, to_dev(phi), to_dev(par), to_dev(hs), 1.0,
                                 fmt=pj.PJ_CSR).cpu().numpy().astype(np.float64)
    ref = oracle.dense_to_csr_values(m, M_ref)
    err = np.abs(M - ref)
    tol = newton_tol(oracle.dense_to_csr_values(m, scale))
    newton_error(M, ref, oracle.dense_to_csr_values(m, scale), f"{name}, {n} states, {layout}")
    assert np.all(err <= tol), float(np.max(err / tol))


def test_default_layout_follows_the_measured_rule(pj, mechs):
    """At most one 32-state tile per SM, and the 53- and 111-species
    Jacobians (but the dense 53-species one) of larger batches, run
    cooperatively; the dense 53-species FP64 Jacobian of a large batch runs
    one state per thread in tensor memory; the 13-species Jacobian of a
    large batch one state per thread in shared memory."""
    import torch
    if torch.cuda.get_device_properties(0).multi_processor_count != 152:
        pytest.skip("the rule was measured on 152-SM parts")
    C, T, P = pj.PJ_LAYOUT_COOP, pj.PJ_LAYOUT_TMEM, pj.PJ_LAYOUT_PERCORE
    h13, h53, h111 = (pj.pj_mech_create(mechs(x)) for x in ("h2co13", "gri53", "usc111"))
    big = 1 << 20
    assert h13.jacobian_layout(pj.PJ_CSR, pj.PJ_F64, 4096) == C
    assert h13.jacobian_layout(pj.PJ_CSR, pj.PJ_F64, big) == P
    assert h53.jacobian_layout(pj.PJ_CSR, pj.PJ_F64, 4096) == C
    assert h53.jacobian_layout(pj.PJ_CSR, pj.PJ_F64, big) == C
    assert h53.jacobian_layout(pj.PJ_CSC, pj.PJ_F64, big) == C
    assert h53.jacobian_layout(pj.PJ_DENSE, pj.PJ_F64, big) == T
    assert h53.jacobian_layout(pj.PJ_CSR, pj.PJ_F32, big) == C
    assert h111.jacobian_layout(pj.PJ_CSR, pj.PJ_F64, big) == C
    assert h111.jacobian_layout(pj.PJ_CSR, pj.PJ_F32, big) == C
    with jacobian_layout("percore"):
        assert h53.jacobian_layout(pj.PJ_CSR, pj.PJ_F64, 4096) == T
    with jacobian_layout("coop"):
        assert h13.jacobian_layout(pj.PJ_CSR, pj.PJ_F64, big) == C
