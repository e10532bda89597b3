"""Host-side failure checks and guard bands, through the C ABI.

* Every entry point whose kernels take a caller-provided workspace returns
  PJ_ERR_NOMEM, launches nothing and leaves its outputs untouched when the
  workspace is one byte short of pj_workspace_size (or missing).
* Every entry point writes only its outputs: each output is allocated with a
  padded leading dimension and a guard band after its last row, both filled
  with a canary value, and after the call every padding column and the guard
  band still hold the canary (out-of-range states, rows or entries would
  overwrite them).  Small batches that end in a ragged last tile.
"""
import numpy as np
import pytest

import synth
from paper_1809_01029_gb300 import _native as N
from tests.parity import jacobian_layout

pytestmark = pytest.mark.gpu

CANARY = {"f64": -7.75e301, "f32": -3.25e38}   # values no evaluation produces
GUARD = 4096


@pytest.fixture(scope="module")
def pj():
    import paper_1809_01029_gb300 as pj
    from paper_1809_01029_gb300 import build
    build.build()
    pj.load_library()
    return pj


class Guarded:
    """A [rows, n] output of leading dimension ld > n inside a larger buffer
    filled with the canary."""

    def __init__(self, rows, n, ld, dtype="f64"):
        import torch
        dt = torch.float64 if dtype == "f64" else torch.float32
        self.rows, self.n, self.ld = rows, n, ld
        self.canary = CANARY[dtype]
        self.big = torch.full((rows * ld + GUARD,), self.canary, dtype=dt, device="cuda")
        self.full = self.big[: rows * ld].view(rows, ld)
        self.t = self.full[:, :n]

    def intact(self):
        import torch
        c = torch.tensor(self.canary, dtype=self.big.dtype, device="cuda")
        pad_ok = bool((self.full[:, self.n:] == c).all()) if self.ld > self.n else True
        return pad_ok and bool((self.big[self.rows * self.ld:] == c).all())


def _states(m, n, ld, mode, seed):
    import torch
    phi, par = synth.make_states(m, n, seed, mode)
    d_phi = torch.full((m.n_species + 1, ld), 1.0, dtype=torch.float64, device="cuda")
    d_phi[:, :n] = torch.from_numpy(phi).cuda()
    return d_phi[:, :n], torch.from_numpy(par).cuda(), phi, par


def _work(torch, nbytes):
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device="cuda")


# (name, op, mechanism, layout): entries whose launch plan uses a workspace
NOMEM_CASES = [
    ("source", "gri53", None),
    ("jacobian", "gri53", "percore"),
    ("jacobian", "usc111", "percore"),   # the cooperative layout needs no workspace
    ("newton", "usc111", "percore"),
    ("eval_y", "ic5874", None),     # up to 112 species y's arrays fit shared memory
    ("vjp", "gri53", None),
    ("fd", "gri53", None),
    ("lu", "ic5874", None),
]


@pytest.mark.parametrize("what,name,layout", NOMEM_CASES)
def test_workspace_one_byte_short_is_rejected(pj, mechs, what, name, layout):
    import contextlib
    import torch
    m = mechs(name)
    h = pj.pj_mech_create(m)
    n = 37 if what != "lu" else 3
    N1 = m.n_species + 1
    op = {"source": pj.PJ_OP_SOURCE, "jacobian": pj.PJ_OP_JACOBIAN, "newton": pj.PJ_OP_NEWTON,
          "eval_y": pj.PJ_OP_Y, "vjp": pj.PJ_OP_VJP, "fd": pj.PJ_OP_FD, "lu": pj.PJ_OP_LU}[what]
    need = h.workspace_size(op, n)
    assert need > 0, "the case must use a workspace"
    phi, par, _, _ = _states(m, n, n, synth.CONP, 71)
    for work, wb in ((_work(torch, need - 1), need - 1), (None, 0)):
        ctx = jacobian_layout(layout) if layout else contextlib.nullcontext()
        outs = []

        def out(rows, dtype="f64"):
            g = Guarded(rows, n, n, dtype)
            outs.append(g)
            return g.t
        with ctx, pytest.raises(pj.PJError) as e:
            if what == "source":
                pj.pj_eval_source_terms(h, synth.CONP, n, par, phi, n, out(N1), None, work, wb)
            elif what == "jacobian":
                pj.pj_eval_jacobian_sparse(h, synth.CONP, pj.PJ_CSR, n, par, phi, n, out(h.nnz), out(N1), None,
                                           work, wb)
            elif what == "newton":
                hs = torch.full((n,), 1e-7, dtype=torch.float64, device="cuda")
                pj.pj_newton_matrix_f32(h, synth.CONP, pj.PJ_CSR, n, par, phi, n, hs, 1.0, out(h.nnz, "f32"),
                                        out(N1), None, work, wb)
            elif what == "eval_y":
                pj.pj_eval_y(h, synth.CONP, n, par, phi, n, out(N1), None, work, wb)
            elif what == "vjp":
                u = torch.ones((m.n_species, n), dtype=torch.float64, device="cuda")
                uT = torch.ones(n, dtype=torch.float64, device="cuda")
                gt = torch.zeros((m.n_reactions, 3), dtype=torch.float64, device="cuda")
                pj.pj_vjp(h, synth.CONP, n, par, phi, n, u, uT, out(N1), out(N1), gt, None, work, wb)
            elif what == "fd":
                pj.pj_eval_jacobian_fd(h, synth.CONP, pj.PJ_CSR, n, par, phi, n, out(h.nnz), out(N1), None,
                                       work, wb)
            else:
                lu_nnz, _ = h.lu_info()
                vals = torch.zeros((h.nnz, n), dtype=torch.float64, device="cuda")
                pj.pj_lu_factor(h, pj.PJ_F64, n, vals, n, out(lu_nnz), None, 1.0, None, work, wb)
        assert e.value.code == N.PJ_ERR_NOMEM, (what, e.value)
        torch.cuda.synchronize()
        assert all(g.intact() and bool((g.t == g.canary).all()) for g in outs), "outputs touched after a rejection"


@pytest.mark.parametrize("name,layout", [("usc111", "coop-global"), ("ic5874", "coop")])
def test_cooperative_workspace_arrays_need_the_workspace(pj, mechs, name, layout):
    """The cooperative layout with its per-state arrays in the workspace (874
    species by default, any mechanism when forced) rejects a call without a
    workspace, launches nothing and leaves the outputs untouched."""
    m = mechs(name)
    h = pj.pj_mech_create(m)
    n = 40
    assert h.workspace_size(pj.PJ_OP_JACOBIAN, n) > 0
    phi, par, _, _ = _states(m, n, n, synth.CONP, 75)
    v, d = Guarded(h.nnz, n, n), Guarded(m.n_species + 1, n, n)
    with jacobian_layout(layout), pytest.raises(pj.PJError) as e:
        pj.pj_eval_jacobian_sparse(h, synth.CONP, pj.PJ_CSR, n, par, phi, n, v.t, d.t, None, None, 0)
    assert e.value.code == N.PJ_ERR_NOMEM
    import torch
    torch.cuda.synchronize()
    assert v.intact() and d.intact() and bool((v.t == v.canary).all())


@pytest.mark.parametrize("layout", ["coop", "coop-global", "percore"])
@pytest.mark.parametrize("name", ["gri53_types", "usc111"])
def test_guard_bands_jacobian_entries(pj, mechs, name, layout):
    """Source terms, CSR / CSC / dense Jacobian and the FP32 Newton matrix of
    a 70-state batch (a ragged last 32-state tile) with ld = n + 9."""
    import torch
    m = mechs(name)
    h = pj.pj_mech_create(m)
    n, ld = 70, 79
    N1 = m.n_species + 1
    for mode in (synth.CONP, synth.CONV):
        phi, par, _, _ = _states(m, n, ld, mode, 73 + mode)
        with jacobian_layout(layout):
            f = Guarded(N1, n, ld)
            pj.source_terms(h, mode, phi, par, out=f.t)
            assert f.intact()
            for fmt in (pj.PJ_CSR, pj.PJ_CSC):
                v, d = Guarded(h.nnz, n, ld), Guarded(N1, n, ld)
                pj.jacobian_sparse(h, mode, phi, par, fmt=fmt, out=v.t, dphi=d.t)
                assert v.intact() and d.intact(), (fmt, mode)
            v, d = Guarded(N1 * N1, n, ld), Guarded(N1, n, ld)
            pj.jacobian_dense(h, mode, phi, par, out=v.t, dphi=d.t)
            assert v.intact() and d.intact(), ("dense", mode)
            hs = torch.full((n,), 1e-8, dtype=torch.float64, device="cuda")
            v, d = Guarded(h.nnz, n, ld, "f32"), Guarded(N1, n, ld)
            pj.newton_matrix_f32(h, mode, phi, par, hs, 1.0, out=v.t, dphi=d.t)
            assert v.intact() and d.intact(), ("newton", mode)
        torch.cuda.synchronize()


def test_guard_bands_forms_fd_noalloc_lu(pj, mechs):
    """y, the VJP, the finite-difference Jacobian, the allocation-free entry
    and the LU factorisation and solve, on a ragged batch with ld = n + 9."""
    import torch
    m = mechs("gri53")
    h = pj.pj_mech_create(m)
    n, ld = 45, 54
    N1 = m.n_species + 1
    phi, par, _, _ = _states(m, n, ld, synth.CONP, 79)
    y = Guarded(N1, n, ld)
    pj.pj_eval_y(h, synth.CONP, n, par, phi, ld, y.t, None, _work(torch, h.workspace_size(pj.PJ_OP_Y, n)),
                 h.workspace_size(pj.PJ_OP_Y, n))
    assert y.intact()
    u = torch.zeros((m.n_species, ld), dtype=torch.float64, device="cuda")[:, :n].normal_()
    uT = torch.ones(n, dtype=torch.float64, device="cuda")
    y2, g = Guarded(N1, n, ld), Guarded(N1, n, ld)
    gt = Guarded(m.n_reactions, 3, 3)
    wb = h.workspace_size(pj.PJ_OP_VJP, n)
    pj.pj_vjp(h, synth.CONP, n, par, phi, ld, u, uT, y2.t, g.t, gt.t, None, _work(torch, wb), wb)
    assert y2.intact() and g.intact() and gt.intact()
    v, d = Guarded(h.nnz, n, ld), Guarded(N1, n, ld)
    wb = h.workspace_size(pj.PJ_OP_FD, n)
    pj.pj_eval_jacobian_fd(h, synth.CONP, pj.PJ_CSR, n, par, phi, ld, v.t, d.t, None, _work(torch, wb), wb)
    assert v.intact() and d.intact()
    v, d = Guarded(h.nnz, n, ld), Guarded(N1, n, ld)
    pj.pj_eval_jacobian_sparse_noalloc(h, synth.CONP, pj.PJ_CSR, n, par, phi, ld, v.t, d.t)
    assert v.intact() and d.intact()
    # LU of M = I - h J (J from the entry above) and a solve
    lu_nnz, _ = h.lu_info()
    lu = Guarded(lu_nnz, n, ld)
    hs = torch.full((n,), 1e-8, dtype=torch.float64, device="cuda")
    wb = h.workspace_size(pj.PJ_OP_LU, n)
    pj.pj_lu_factor(h, pj.PJ_F64, n, v.t, ld, lu.t, hs, 1.0, None, _work(torch, wb), wb)
    assert lu.intact()
    b = torch.zeros((N1, ld), dtype=torch.float64, device="cuda")[:, :n].normal_()
    x = Guarded(N1, n, ld)
    pj.pj_lu_solve(h, pj.PJ_F64, n, lu.t, ld, b, x.t)
    torch.cuda.synchronize()
    assert x.intact()
