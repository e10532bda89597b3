"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/pyjac_gb.h, builds the exact sparsity pattern and rejects
bad arguments with the documented codes."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
import synth
import paper_1809_01029_gb300 as pj
from paper_1809_01029_gb300 import _native as N
from tests import tiny_mechs as tm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1809_01029_gb300 import build
    build.build()
    return N.load()


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pj_\w+)\s*\(", src, re.M))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_every_declared_symbol_has_a_binding_signature(lib):
    missing = [n for n in declared_symbols() if n not in N.SIGNATURES]
    assert not missing, missing


def test_version(lib):
    assert b"pyjac_gb" in lib.pj_version()


@pytest.mark.parametrize("name", ["h2co13", "gri53", "gri53_types", "usc111"])
def test_pattern_bit_exact_against_oracle(lib, mechs, name):
    m = mechs(name)
    h = pj.pj_mech_create(m)
    for fmt, ref in ((pj.PJ_CSR, oracle.csr_pattern(m)), (pj.PJ_CSC, oracle.csc_pattern(m))):
        ptr, idx = h.sparsity(fmt)
        assert ptr.tobytes() == ref[0].astype(np.int32).tobytes()
        assert idx.tobytes() == ref[1].astype(np.int32).tobytes()


@pytest.mark.parametrize("mk", ["all_kinds", "bath_efficiency"])
def test_pattern_tiny_mechanisms(lib, mk):
    m = getattr(tm, mk)()
    h = pj.pj_mech_create(m)
    ptr, idx = h.sparsity(pj.PJ_CSR)
    rp, ci = oracle.csr_pattern(m)
    assert np.array_equal(ptr, rp) and np.array_equal(idx, ci)


@pytest.mark.parametrize("name", ["gri53", "gri53_types"])
def test_mechanism_file_round_trip(lib, mechs, tmp_path, name):
    m = mechs(name)
    path = str(tmp_path / f"{name}.pjmech")
    synth.write_mechanism(m, path)
    back = synth.read_mechanism(path)
    for f in ("W", "nasa_low", "nasa_high", "kind", "reversible", "A", "beta", "Ea", "A0", "troe", "sri",
              "eff_val", "chem", "rev_explicit", "rev_arr", "plog_ptr", "plog", "cheb_ptr", "cheb_shape",
              "cheb_range", "cheb_coef"):
        assert np.array_equal(getattr(m, f), getattr(back, f)), f
    h1 = pj.pj_mech_create(m)
    h2 = pj.pj_mech_load(path)
    assert (h1.n_species, h1.n_reactions, h1.nnz) == (h2.n_species, h2.n_reactions, h2.nnz)
    for fmt in (pj.PJ_CSR, pj.PJ_CSC):
        a, b = h1.sparsity(fmt), h2.sparsity(fmt)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_corrupt_mechanism_file(lib, tmp_path, mechs):
    path = str(tmp_path / "bad.pjmech")
    synth.write_mechanism(mechs("h2co13"), path)
    txt = open(path).read().split("\n")
    open(path, "w").write("\n".join(txt[: len(txt) // 2]))
    with pytest.raises(pj.PJError) as e:
        pj.pj_mech_load(path)
    assert e.value.code == N.PJ_ERR_MECH
    with pytest.raises(pj.PJError) as e:
        pj.pj_mech_load(str(tmp_path / "missing"))
    assert e.value.code == N.PJ_ERR_ARG


def test_invalid_mechanisms_rejected(lib):
    base = tm.all_kinds()
    cases = []
    m = base.copy(); m.A = m.A.copy(); m.A[0] = -1.0; cases.append(m)
    m = base.copy(); m.reac_sp = m.reac_sp.copy(); m.reac_sp[0, 0] = 99; cases.append(m)
    m = base.copy(); m.kind = m.kind.copy(); m.kind[0] = 9; cases.append(m)
    m = base.copy(); m.troe_n = m.troe_n.copy(); m.troe_n[int(np.flatnonzero(m.kind == synth.TROE)[0])] = 5
    cases.append(m)
    for bad in cases:
        with pytest.raises(pj.PJError) as e:
            pj.pj_mech_create(bad)
        assert e.value.code == N.PJ_ERR_MECH


def test_argument_errors(lib):
    h = pj.pj_mech_create(tm.all_kinds())
    f = lib.pj_eval_source_terms
    p = C.c_void_p(16)
    assert f(None, 0, 1, p, p, 1, p, None, None, 0, None) == N.PJ_ERR_ARG
    assert f(h.handle, 7, 1, p, p, 1, p, None, None, 0, None) == N.PJ_ERR_ARG
    assert f(h.handle, 0, 4, p, p, 2, p, None, None, 0, None) == N.PJ_ERR_ARG       # ld < n
    assert f(h.handle, 0, -1, p, p, 2, p, None, None, 0, None) == N.PJ_ERR_ARG
    assert f(h.handle, 0, 4, None, p, 4, p, None, None, 0, None) == N.PJ_ERR_ARG
    g = lib.pj_eval_jacobian_sparse
    assert g(h.handle, 0, 2, 1, p, p, 1, p, None, None, None, 0, None) == N.PJ_ERR_ARG  # fmt
    hh = lib.pj_eval_jacobian_sparse_host
    assert hh(h.handle, 0, 2, 1, p, p, p, p, None, 0, None) == N.PJ_ERR_ARG              # fmt
    assert hh(h.handle, 0, 0, 1, p, p, p, p, None, -5, None) == N.PJ_ERR_ARG             # chunk < 0
    assert hh(h.handle, 0, 0, 1, p, p, p, None, None, 0, None) == N.PJ_ERR_ARG           # no h_dphi
    assert lib.pj_workspace_size(h.handle, 99, 10, C.byref(C.c_size_t())) == N.PJ_ERR_ARG
    assert b"fmt" in lib.pj_last_error() or len(lib.pj_last_error()) > 0


def test_no_device_means_no_silent_fallback(lib):
    """Without a GPU the evaluation entry points fail; nothing computes on the host."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("GPU present")
    except ImportError:
        pass
    h = pj.pj_mech_create(tm.all_kinds())
    p = C.c_void_p(16)
    rc = lib.pj_eval_source_terms(h.handle, 0, 1, p, p, 1, p, None, None, 0, None)
    assert rc == N.PJ_ERR_CUDA
    rc = lib.pj_eval_jacobian_sparse_host(h.handle, 0, 0, 1, p, p, p, p, None, 0, None)
    assert rc == N.PJ_ERR_CUDA


@pytest.mark.parametrize("name", ["all_kinds", "bath_efficiency", "all_types", "h2co13", "gri53", "gri53_types", "usc111",
                                  "ic5874"])
def test_approximate_pattern_bit_exact_against_oracle(lib, mechs, name):
    """The approximate Jacobian form (Sec. 3.4) has its own, sparser pattern."""
    m = getattr(tm, name)() if name in ("all_kinds", "bath_efficiency", "all_types") else mechs(name)
    h = pj.pj_mech_create(m)
    ha = h.with_jacobian_form(pj.PJ_JAC_APPROX)
    assert (h.jacobian_form, ha.jacobian_form) == (pj.PJ_JAC_EXACT, pj.PJ_JAC_APPROX)
    assert ha.nnz == int(oracle.sparsity_pattern(m, oracle.APPROX).sum()) <= h.nnz
    for fmt, ref in ((pj.PJ_CSR, oracle.csr_pattern(m, oracle.APPROX)),
                     (pj.PJ_CSC, oracle.csc_pattern(m, oracle.APPROX))):
        ptr, idx = ha.sparsity(fmt)
        assert ptr.tobytes() == ref[0].astype(np.int32).tobytes()
        assert idx.tobytes() == ref[1].astype(np.int32).tobytes()
    back = ha.with_jacobian_form(pj.PJ_JAC_EXACT)
    assert back.nnz == h.nnz and np.array_equal(back.sparsity(pj.PJ_CSR)[1], h.sparsity(pj.PJ_CSR)[1])


def test_jacobian_form_rejects_unknown_form(lib, mechs):
    h = pj.pj_mech_create(mechs("h2co13"))
    out = C.c_void_p()
    assert lib.pj_mech_with_jacobian_form(h.handle, 7, C.byref(out)) == N.PJ_ERR_ARG
    assert lib.pj_mech_with_jacobian_form(None, 0, C.byref(out)) == N.PJ_ERR_ARG


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("name", ["all_kinds", "bath_efficiency", "all_types", "h2co13", "gri53", "gri53_types",
                                  "usc111"])
def test_lu_ordering_and_pattern_bit_exact_against_oracle(lib, mechs, name, form):
    """The Newton-matrix LU's symbolic phase (pivot order, fill, storage
    order) is index work: identical to the oracle's."""
    m = getattr(tm, name)() if name in ("all_kinds", "bath_efficiency", "all_types") else mechs(name)
    h = pj.pj_mech_create(m)
    if form:
        h = h.with_jacobian_form(pj.PJ_JAC_APPROX)
    perm, F, (r, c) = oracle.linalg.lu_symbolic(m, oracle.APPROX if form else oracle.EXACT)
    k, p = h.lu_info()
    hr, hc = h.lu_pattern()
    assert k == len(r) == F.sum()
    assert p.tobytes() == perm.astype(np.int32).tobytes()
    assert hr.tobytes() == r.tobytes() and hc.tobytes() == c.tobytes()


def test_lu_ordering_and_pattern_874_species(lib, mechs):
    m = mechs("ic5874")
    h = pj.pj_mech_create(m)
    perm, F, (r, c) = oracle.linalg.lu_symbolic(m)
    k, p = h.lu_info()
    hr, hc = h.lu_pattern()
    assert k == len(r) and np.array_equal(p, perm) and np.array_equal(hr, r) and np.array_equal(hc, c)


def test_arrhenius_parameters_round_trip(lib, mechs):
    """pj_mech_arrhenius returns (ln A, beta, Ea) in reaction order;
    pj_mech_with_arrhenius makes a new handle with them replaced and leaves
    the source handle as it was; non-finite parameters are rejected."""
    m = mechs("gri53_types")
    h = pj.pj_mech_create(m)
    a, b, e = h.arrhenius()
    assert np.array_equal(a, np.log(m.A)) and np.array_equal(b, m.beta) and np.array_equal(e, m.Ea)
    rng = np.random.default_rng(5)
    a2, b2, e2 = a + rng.normal(0, 0.1, a.shape), b + 0.05, e * 1.01
    h2 = pj.pj_mech_with_arrhenius(h, a2, b2, e2)
    got = h2.arrhenius()
    assert np.allclose(got[0], a2, rtol=0, atol=4e-15 * np.abs(a2).max()) and np.array_equal(got[1], b2)
    assert np.array_equal(got[2], e2)
    assert np.array_equal(h.arrhenius()[0], a)
    assert h2.nnz == h.nnz and h2.jacobian_form == h.jacobian_form
    bad = a2.copy()
    bad[3] = np.nan
    with pytest.raises(pj.PJError) as err:
        h.with_arrhenius(bad, b2, e2)
    assert err.value.code == N.PJ_ERR_ARG
    with pytest.raises(ValueError):
        h.with_arrhenius(a2[:-1], b2, e2)
