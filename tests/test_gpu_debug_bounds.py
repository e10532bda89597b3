"""The bounds-checked build (compiled with PJ_DEBUG_BOUNDS): every lookup in
an index table derived at mechanism load is checked before use into a
device error word, with no trap.

Every entry point runs on the tiny mechanisms (every reaction kind, the
bath-gas cases of Sec. 3.4's pattern rules, every less common type) and the
53-species all-types mechanism with the word staying 0; then a target-list
entry is set out of range through the build's test hook and the Jacobian
evaluations record it in the word (bit 1) instead of writing out of range.
Runs in a fresh process that loads libpyjac_gb_dbg.so (PYJAC_GB_LIB)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, os, sys
import numpy as np
import torch
sys.path.insert(0, os.environ["PJ_ROOT"])
import synth
from tests import tiny_mechs as tm
import paper_1809_01029_gb300 as pj
assert pj.pj_debug_build()
res = {}
def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()
for name in ("all_kinds", "bath_efficiency", "all_types", "gri53_types"):
    m = getattr(tm, name)() if name != "gri53_types" else synth.make_mechanism(name)
    h = pj.pj_mech_create(m)
    ha = h.with_jacobian_form(pj.PJ_JAC_APPROX)
    n = 45
    N1 = m.n_species + 1
    words = []
    for mode in (synth.CONP, synth.CONV):
        phi, par = synth.make_states(m, n, 17 + mode, mode)
        d_phi, d_par = dev(phi), dev(par)
        hs = torch.full((n,), 1e-8, dtype=torch.float64, device="cuda")
        for lay in ("coop", "percore"):
            os.environ["PYJAC_GB_JAC_LAYOUT"] = lay
            for hh in (h, ha):
                for fmt in (pj.PJ_CSR, pj.PJ_CSC):
                    pj.jacobian_sparse(hh, mode, d_phi, d_par, fmt=fmt)
                    pj.newton_matrix_f32(hh, mode, d_phi, d_par, hs, 1.0, fmt=fmt)
                pj.jacobian_dense(hh, mode, d_phi, d_par)
                pj.newton_matrix_f32(hh, mode, d_phi, d_par, hs, 1.0, fmt=pj.PJ_DENSE)
        os.environ.pop("PYJAC_GB_JAC_LAYOUT")
        pj.source_terms(h, mode, d_phi, d_par)
        pj.eval_y(h, mode, d_phi, d_par)
        uw, uT = synth.make_cotangents(m.n_species, n, 3)
        pj.vjp(h, mode, d_phi, d_par, dev(uw), dev(uT))
        pj.jacobian_fd(h, mode, d_phi, d_par)
        v = torch.empty((h.nnz, n), dtype=torch.float64, device="cuda")
        f = torch.empty((N1, n), dtype=torch.float64, device="cuda")
        pj.pj_eval_jacobian_sparse_noalloc(h, mode, pj.PJ_CSR, n, d_par, d_phi, n, v, f)
        lu = pj.lu_factor(h, pj.jacobian_sparse(h, mode, d_phi, d_par), h=hs)
        pj.lu_solve(h, lu, torch.ones((N1, n), dtype=torch.float64, device="cuda"))
        batches = [(d_par[:20], d_phi[:, :20].contiguous(), torch.empty((h.nnz, 20), dtype=torch.float64,
                    device="cuda"), torch.empty((N1, 20), dtype=torch.float64, device="cuda"))]
        pj.Plan(h, pj.PJ_OP_JACOBIAN, mode, batches).run()
        torch.cuda.synchronize()
        words.append(pj.pj_debug_word(h, clear=True))
        words.append(pj.pj_debug_word(ha, clear=True))
    res[name] = words
# a target-list entry out of range: recorded, not written
m = tm.all_kinds()
h = pj.pj_mech_create(m)
phi, par = synth.make_states(m, 40, 5, synth.CONP)
caught = {}
for lay in ("coop", "percore"):
    os.environ["PYJAC_GB_JAC_LAYOUT"] = lay
    pj.pj_debug_set_target(h, pj.PJ_CSR, 0, 1 << 28)
    out = pj.jacobian_sparse(h, synth.CONP, dev(phi), dev(par), fmt=pj.PJ_CSR)
    torch.cuda.synchronize()
    caught[lay] = pj.pj_debug_word(h, clear=True)
res["corrupt_target"] = caught
print("RESULT " + json.dumps(res))
'''


def test_bounds_checked_build_clean_and_catches_a_corrupt_target_list():
    from paper_1809_01029_gb300 import build
    lib = build.build(debug_bounds=True)
    env = dict(os.environ, PYJAC_GB_LIB=lib, PJ_ROOT=ROOT)
    env.pop("PYJAC_GB_JAC_LAYOUT", None)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, cwd=ROOT, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    for name, words in res.items():
        if name != "corrupt_target":
            assert all(w == 0 for w in words), (name, words)
    for lay, w in res["corrupt_target"].items():
        assert w & 1, (lay, w)          # the target-list bit
