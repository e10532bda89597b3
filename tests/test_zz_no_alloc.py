"""The allocation-free Jacobian entry point against the regular one.

pj_eval_jacobian_sparse_noalloc serves callers that cannot allocate device
memory (and so cannot pass a workspace): it keeps its scratch in a fixed
device array inside the library.  This test calls it twice in a row through
the C ABI — the second call runs on whatever the first left in that shared
array — and checks both results against the regular entry point, which
takes a caller-allocated workspace.  It lives in its own file so that pytest
collects it after every other test.
"""
import numpy as np
import pytest

import synth
from tests.parity import RTOL_SRC, ATOL_SRC, RTOL_JAC, ATOL_JAC, check_close, jacobian_layout

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,n,mode,fmt", [
    ("usc111", 700, synth.CONP, 0),    # large enough that the regular path uses a workspace
    ("usc111", 333, synth.CONV, 1),
    ("gri53", 1500, synth.CONP, 0),    # regular path keeps its arrays in shared memory
])
def test_noalloc_matches_regular_entry_point_on_two_calls(mechs, name, n, mode, fmt):
    import torch
    import paper_1809_01029_gb300 as pj
    from paper_1809_01029_gb300 import build
    build.build()
    m = mechs(name)
    h = pj.pj_mech_create(m)
    phi, par = synth.make_states(m, n, 4242 + n, mode)
    d_phi = torch.from_numpy(phi).cuda()
    d_par = torch.from_numpy(par).cuda()
    N1 = m.n_species + 1

    wb = h.workspace_size(pj.PJ_OP_JACOBIAN, n)
    work = torch.empty(max(wb, 1), dtype=torch.uint8, device="cuda")
    ref = torch.empty((h.nnz, n), dtype=torch.float64, device="cuda")
    ref_f = torch.empty((N1, n), dtype=torch.float64, device="cuda")
    # the regular entry's one-state-per-thread layout runs the same arithmetic
    # in the same order as this entry point
    with jacobian_layout("percore"):
        pj.pj_eval_jacobian_sparse(h, mode, fmt, n, d_par, d_phi, n, ref, ref_f, None, work, wb)
    ref = ref.cpu().numpy()
    ref_f = ref_f.cpu().numpy()
    assert np.all(np.isfinite(ref))

    for call in range(2):
        vals = torch.full((h.nnz, n), float("nan"), dtype=torch.float64, device="cuda")
        f = torch.full((N1, n), float("nan"), dtype=torch.float64, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        pj.pj_eval_jacobian_sparse_noalloc(h, mode, fmt, n, d_par, d_phi, n, vals, f, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        check_close(vals.cpu().numpy(), ref, np.abs(ref), RTOL_JAC, ATOL_JAC, f"{name} call {call} Jacobian")
        check_close(f.cpu().numpy(), ref_f, np.abs(ref_f), RTOL_SRC, ATOL_SRC, f"{name} call {call} source terms")
