"""GPU parity of source terms and Jacobians against the CPU oracle, through
the C ABI (the Python binding only marshals arguments)."""
import numpy as np
import pytest

import oracle
import synth
from tests import tiny_mechs as tm
from tests.parity import RTOL_SRC, ATOL_SRC, RTOL_JAC, ATOL_JAC, check_close, paper_error_norms, jacobian_layout

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


def to_dev(a, ld=None):
    import torch
    a = np.asarray(a, dtype=np.float64)
    if ld is None or a.ndim == 1:
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    buf = torch.full((a.shape[0], ld), float("nan"), dtype=torch.float64, device="cuda")
    buf[:, : a.shape[1]] = torch.from_numpy(a).cuda()
    return buf[:, : a.shape[1]]


SRC_CASES = [("all_kinds", 37), ("bath_efficiency", 33), ("all_types", 41), ("h2co13", 4096), ("gri53", 777), ("gri53_types", 333),
               ("usc111", 301)]


@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
@pytest.mark.parametrize("name,n", SRC_CASES)
def test_source_terms_match_oracle(pj, mechs, name, n, mode):
    m = _mech(mechs, name)
    h = pj.pj_mech_create(m)
    phi, par = synth.make_states(m, n, 100 + n, mode)
    out = pj.source_terms(h, mode, to_dev(phi, ld=n + 3), to_dev(par)).cpu().numpy()
    ref, env = oracle.source_term_envelope(m, mode, phi, par)
    check_close(out, ref, env, RTOL_SRC, ATOL_SRC, f"{name} mode={mode}")


JAC_CASES = [("all_kinds", 40), ("bath_efficiency", 35), ("all_types", 36), ("h2co13", 200), ("gri53", 70), ("gri53_types", 45),
             ("usc111", 20)]


@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
@pytest.mark.parametrize("name,n", JAC_CASES)
def test_jacobian_all_formats_match_oracle(pj, mechs, name, n, mode):
    import torch
    m = _mech(mechs, name)
    h = pj.pj_mech_create(m)
    phi, par = synth.make_states(m, n, 300 + n, mode)
    J, env = oracle.jacobian_envelope(m, mode, phi, par)
    f_ref, f_env = oracle.source_term_envelope(m, mode, phi, par)
    dphi = torch.empty((m.n_species + 1, n), dtype=torch.float64, device="cuda")
    d_phi, d_par = to_dev(phi), to_dev(par)
    # dense
    N1 = m.n_species + 1
    Jd = pj.jacobian_dense(h, mode, d_phi, d_par, dphi=dphi).cpu().numpy().reshape(N1, N1, n)
    check_close(Jd, J, env, RTOL_JAC, ATOL_JAC, f"{name} dense mode={mode}")
    check_close(dphi.cpu().numpy(), f_ref, f_env, RTOL_SRC, ATOL_SRC, f"{name} f from jacobian kernel")
    mask = oracle.sparsity_pattern(m)
    assert np.all(Jd[~mask] == 0.0)
    # CSR / CSC values in the order of pj_sparsity
    for fmt, conv in ((pj.PJ_CSR, oracle.dense_to_csr_values), (pj.PJ_CSC, oracle.dense_to_csc_values)):
        vals = pj.jacobian_sparse(h, mode, d_phi, d_par, fmt=fmt).cpu().numpy()
        check_close(vals, conv(m, J), conv(m, env), RTOL_JAC, ATOL_JAC, f"{name} fmt={fmt} mode={mode}")
    # the paper's norms (Sec. 3.3): LAPACK-style E_L, and the filtered E_C at
    # the relaxed threshold C = 1e15 against the largest value the paper
    # reports for its own Jacobians at that threshold (4.5e-5)
    EL, EC = paper_error_norms(Jd, J, C_thresh=1e15)
    assert EL < 1e-10
    assert EC < 4.5e-5, EC


def test_invalid_states_give_nan_and_count(pj, mechs):
    import torch
    m = mechs("h2co13")
    h = pj.pj_mech_create(m)
    n = 64
    phi, par = synth.make_states(m, n, 5, synth.CONP)
    phi[0, 3] = -10.0                     # T <= 0
    phi[4, 7] = np.nan                    # non-finite species amount
    phi[2:, 11] *= 1.5                    # sum of species above the total: bath gas < 0
    par[20] = 0.0                         # P <= 0
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = pj.source_terms(h, synth.CONP, to_dev(phi), to_dev(par), status=status).cpu().numpy()
    assert int(status.item()) == 4
    bad = [3, 7, 11, 20]
    assert np.all(np.isnan(out[:, bad]))
    good = np.setdiff1d(np.arange(n), bad)
    ref, env = oracle.source_term_envelope(m, synth.CONP, phi[:, good], par[good])
    check_close(out[:, good], ref, env, RTOL_SRC, ATOL_SRC, "valid neighbours of invalid states")
    status.zero_()
    vals = pj.jacobian_sparse(h, synth.CONP, to_dev(phi), to_dev(par), status=status).cpu().numpy()
    assert int(status.item()) == 4 and np.all(np.isnan(vals[:, bad]))
    assert np.all(np.isfinite(vals[:, good]))


def test_empty_and_single_state(pj, mechs):
    import torch
    m = mechs("h2co13")
    h = pj.pj_mech_create(m)
    phi, par = synth.make_states(m, 1, 9, synth.CONV)
    out = pj.source_terms(h, synth.CONV, to_dev(phi), to_dev(par)).cpu().numpy()
    ref, env = oracle.source_term_envelope(m, synth.CONV, phi, par)
    check_close(out, ref, env, RTOL_SRC, ATOL_SRC, "single state")
    e = torch.empty((m.n_species + 1, 0), dtype=torch.float64, device="cuda")
    pj.pj_eval_source_terms(h, synth.CONV, 0, e[0], e, 1, e)


def test_state_at_T_mid_and_boundaries(pj, mechs):
    """T exactly at the NASA range switch and at both ends of the workload range."""
    m = mechs("gri53")
    h = pj.pj_mech_create(m)
    Ts = [1000.0, np.nextafter(1000.0, 0), 600.0, 2500.0, 300.0, 3400.0]
    cols = [synth.make_states(m, 1, 77 + i, synth.CONP, T_range=(T, T)) for i, T in enumerate(Ts)]
    phi = np.concatenate([c[0] for c in cols], axis=1)
    par = np.concatenate([c[1] for c in cols])
    assert np.array_equal(phi[0], Ts)
    out = pj.source_terms(h, synth.CONP, to_dev(phi), to_dev(par)).cpu().numpy()
    ref, env = oracle.source_term_envelope(m, synth.CONP, phi, par)
    check_close(out, ref, env, RTOL_SRC, ATOL_SRC, "T boundaries")
    J, jenv = oracle.jacobian_envelope(m, synth.CONP, phi, par)
    vals = pj.jacobian_sparse(h, synth.CONP, to_dev(phi), to_dev(par)).cpu().numpy()
    check_close(vals, oracle.dense_to_csr_values(m, J), oracle.dense_to_csr_values(m, jenv), RTOL_JAC, ATOL_JAC,
                "T boundaries jacobian")


@pytest.mark.parametrize("layout", ["percore", "coop"])
def test_sharding_by_offset_equals_one_launch(pj, mechs, layout):
    """Replicas-only multi-GPU: a shard is (pointer offset, n).  Evaluating a
    batch shard by shard gives the same bits as one launch with the
    one-state-per-thread layout; with the cooperative layout (cross-warp
    reductions in any order) the same values to the rounding of the sums,
    checked against the oracle's envelope on every 25th state."""
    import torch
    m = mechs("gri53")
    h = pj.pj_mech_create(m)
    n = 1000
    phi, par = synth.make_states(m, n, 31, synth.CONP)
    d_phi, d_par = to_dev(phi), to_dev(par)
    with jacobian_layout(layout):
        whole = pj.jacobian_sparse(h, synth.CONP, d_phi, d_par)
        parts = []
        for lo, hi in ((0, 333), (333, 640), (640, 1000)):
            parts.append(pj.jacobian_sparse(h, synth.CONP, d_phi[:, lo:hi], d_par[lo:hi]))
    cat = torch.cat(parts, dim=1)
    if layout == "percore":
        assert torch.equal(whole, cat)
        return
    pick = np.arange(0, n, 25)
    J, env = oracle.jacobian_envelope(m, synth.CONP, phi[:, pick], par[pick])
    ref, env = oracle.dense_to_csr_values(m, J), oracle.dense_to_csr_values(m, env)
    for got, what in ((whole, "one launch"), (cat, "shards")):
        check_close(got.cpu().numpy()[:, pick], ref, env, RTOL_JAC, ATOL_JAC, what)
    check_close(cat.cpu().numpy()[:, pick], whole.cpu().numpy()[:, pick], env, 1e-13, 0.0, "shards vs one launch")


def test_jacobian_requires_source_term_buffer(pj, mechs):
    import torch
    from paper_1809_01029_gb300 import _native as N
    m = mechs("h2co13")
    h = pj.pj_mech_create(m)
    phi, par = synth.make_states(m, 8, 1, synth.CONP)
    d_phi, d_par = to_dev(phi), to_dev(par)
    vals = torch.empty((h.nnz, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(pj.PJError) as e:
        pj.pj_eval_jacobian_sparse(h, synth.CONP, pj.PJ_CSR, 8, d_par, d_phi, 8, vals, None)
    assert e.value.code == N.PJ_ERR_ARG


def test_mechanism_file_gives_identical_results(pj, mechs, tmp_path):
    """A mechanism loaded from its text file evaluates bit for bit like the
    one created from arrays (every reaction type)."""
    import torch
    m = mechs("gri53_types")
    path = str(tmp_path / "types.pjmech")
    synth.write_mechanism(m, path)
    h1, h2 = pj.pj_mech_create(m), pj.pj_mech_load(path)
    for mode in (synth.CONP, synth.CONV):
        phi, par = synth.make_states(m, 300, 4 + mode, mode)
        d_phi, d_par = to_dev(phi), to_dev(par)
        assert torch.equal(pj.source_terms(h1, mode, d_phi, d_par), pj.source_terms(h2, mode, d_phi, d_par))
        with jacobian_layout("percore"):  # bit-reproducible layout
            assert torch.equal(pj.jacobian_sparse(h1, mode, d_phi, d_par), pj.jacobian_sparse(h2, mode, d_phi, d_par))


@pytest.mark.parametrize("fmt", ["csr", "csc"])
def test_host_buffer_entry_equals_device_entry(pj, mechs, fmt):
    """pj_eval_jacobian_sparse_host (host buffers, chunked and overlapped
    transfers) gives the device entry's bits (both with the bit-reproducible
    one-state-per-thread layout): several chunks with a ragged last one from
    page-locked buffers, one chunk from pageable numpy arrays, and the
    invalid-state count."""
    with jacobian_layout("percore"):
        _host_entry_case(pj, mechs, fmt)


def test_host_buffer_entry_cooperative_layout(pj, mechs):
    """The host-buffer entry with the default (cooperative) layout: the same
    NaN pattern and invalid-state count as the device entry, values against
    the oracle on sampled states of every chunk."""
    import torch
    m = mechs("gri53")
    h = pj.pj_mech_create(m)
    n = 3000
    phi, par = synth.make_states(m, n, 62, synth.CONP)
    phi[0, 2100] = -1.0
    with jacobian_layout("coop"):
        vals, dphi, bad = pj.jacobian_sparse_host(h, synth.CONP, torch.from_numpy(phi), torch.from_numpy(par),
                                                  chunk=1024)
    assert bad == 1
    vals, dphi = vals.numpy(), dphi.numpy()
    assert np.isnan(vals[:, 2100]).all() and np.isnan(dphi[:, 2100]).all()
    pick = np.array([0, 511, 1023, 1024, 1500, 2047, 2048, 2999])
    J, env = oracle.jacobian_envelope(m, synth.CONP, phi[:, pick], par[pick])
    check_close(vals[:, pick], oracle.dense_to_csr_values(m, J), oracle.dense_to_csr_values(m, env), RTOL_JAC,
                ATOL_JAC, "host entry, cooperative layout")
    f_ref, f_env = oracle.source_term_envelope(m, synth.CONP, phi[:, pick], par[pick])
    check_close(dphi[:, pick], f_ref, f_env, RTOL_SRC, ATOL_SRC, "host entry source terms")


def _host_entry_case(pj, mechs, fmt):
    import torch
    m = mechs("gri53")
    h = pj.pj_mech_create(m)
    f = pj.PJ_CSR if fmt == "csr" else pj.PJ_CSC
    n = 5000
    phi, par = synth.make_states(m, n, 61, synth.CONP)
    phi[0, 4321] = -1.0                                   # one invalid state
    ref = pj.jacobian_sparse(h, synth.CONP, to_dev(phi), to_dev(par), fmt=f).cpu().numpy()
    ref_f = torch.empty((m.n_species + 1, n), dtype=torch.float64, device="cuda")
    pj.jacobian_sparse(h, synth.CONP, to_dev(phi), to_dev(par), fmt=f, dphi=ref_f)
    ref_f = ref_f.cpu().numpy()
    vals, dphi, bad = pj.jacobian_sparse_host(h, synth.CONP, torch.from_numpy(phi), torch.from_numpy(par), fmt=f,
                                              chunk=1024)
    assert bad == 1
    assert np.array_equal(vals.numpy(), ref, equal_nan=True)
    assert np.array_equal(dphi.numpy(), ref_f, equal_nan=True)
    v2 = np.full((h.nnz, n), 7.0)
    d2 = np.full((m.n_species + 1, n), 7.0)
    assert pj.pj_eval_jacobian_sparse_host(h, synth.CONP, f, n, par, phi, v2, d2) == 1
    assert np.array_equal(v2, ref, equal_nan=True) and np.array_equal(d2, ref_f, equal_nan=True)
