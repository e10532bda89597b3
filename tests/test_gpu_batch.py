"""Batching form: plans of uneven batches through persistent kernels, CUDA
graph capture and replay, grouped launches, and the autotuner."""
import os

import numpy as np
import pytest

import oracle
import synth
from tests.parity import RTOL_SRC, ATOL_SRC, RTOL_JAC, ATOL_JAC, check_close, jacobian_layout

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def percore_entry_points():
    """The plans' persistent kernels evaluate one state per thread, as the
    direct entry points' "percore" layout does: the same arithmetic, in
    other kernels, whose multiply-adds the compiler contracts on its own, so
    the two agree to the last bits of rounding (same_bits_but_rounding)."""
    with jacobian_layout("percore"):
        yield


def same_bits_but_rounding(o, r, rel=1e-13):
    """o and r (entries x states) equal to within rel of each state's largest
    entry: one state per thread in two kernels (a plan's and an entry
    point's) differs by the rounding of single operations, nothing more."""
    import torch
    if torch.equal(o, r):
        return True
    scale = torch.maximum(o.abs(), r.abs()).amax(dim=0, keepdim=True)
    return bool(((o - r).abs() <= rel * scale).all())


@pytest.fixture(scope="module")
def pj():
    import paper_1809_01029_gb300 as pj
    from paper_1809_01029_gb300 import build
    build.build()
    pj.load_library()
    return pj


def make_batches(torch, m, sizes, seed, mode, op, nnz):
    out = []
    for b, n in enumerate(sizes):
        phi, par = synth.make_states(m, max(n, 1), seed + b, mode)
        phi, par = phi[:, :n], par[:n]
        d_phi = torch.from_numpy(np.ascontiguousarray(phi)).cuda()
        d_par = torch.from_numpy(np.ascontiguousarray(par)).cuda()
        rows = nnz if op == 1 else m.n_species + 1
        o = torch.full((rows, max(n, 1)), float("nan"), dtype=torch.float64, device="cuda")[:, :n]
        f = torch.full((m.n_species + 1, max(n, 1)), float("nan"), dtype=torch.float64, device="cuda")[:, :n]
        out.append((d_par, d_phi, o, f))
    return out


SIZES = [1, 31, 33, 0, 500, 1000, 77]


@pytest.mark.parametrize("mode", [synth.CONP, synth.CONV])
def test_plan_matches_single_batch_entry_points(pj, mechs, mode):
    import torch
    m = mechs("gri53")
    h = pj.pj_mech_create(m)
    bj = make_batches(torch, m, SIZES, 50, mode, 1, h.nnz)
    plan = pj.Plan(h, pj.PJ_OP_JACOBIAN, mode, bj, fmt=pj.PJ_CSR)
    plan.run()
    bs = make_batches(torch, m, SIZES, 50, mode, 0, h.nnz)
    plan_s = pj.Plan(h, pj.PJ_OP_SOURCE, mode, bs)
    plan_s.run()
    torch.cuda.synchronize()
    for (par, phi, o, f), (_, _, osrc, _) in zip(bj, bs):
        n = phi.shape[1]
        if n == 0:
            continue
        ref = pj.jacobian_sparse(h, mode, phi, par, fmt=pj.PJ_CSR)
        ref_f = pj.source_terms(h, mode, phi, par)
        assert same_bits_but_rounding(o, ref)
        assert same_bits_but_rounding(osrc, ref_f)
        check_close(f.cpu().numpy(), ref_f.cpu().numpy(), np.abs(ref_f.cpu().numpy()), RTOL_SRC, ATOL_SRC, "dphi")


@pytest.mark.parametrize("name", ["gri53", "usc111"])
def test_cooperative_plan_shapes(pj, mechs, name):
    """The cooperative shapes of a plan (arrays in shared memory and in the
    workspace, 16 and 8 warps) on uneven batches, and a graph replay: within
    rounding of the one-state-per-thread entry (several warps sum into one
    entry), and a sample of every batch against the oracle."""
    import torch
    m = mechs(name)
    h = pj.pj_mech_create(m)
    sizes = [1, 31, 33, 0, 300, 77]
    bj = make_batches(torch, m, sizes, 95, synth.CONV, 1, h.nnz)
    refs = [pj.jacobian_sparse(h, synth.CONV, phi, par).clone() if phi.shape[1] else None for (par, phi, _, _) in bj]
    st = torch.cuda.Stream()
    plan = pj.Plan(h, pj.PJ_OP_JACOBIAN, synth.CONV, bj, max_states_per_launch=200)
    for shape in ((512, 1, 1), (512, 1, 0), (256, 2, 0)):
        plan.set_config(*shape)
        with torch.cuda.stream(st):
            plan.capture(st)
            for (_, _, o, f) in bj:
                o.fill_(float("nan"))
                f.fill_(float("nan"))
            plan.launch(st)
        st.synchronize()
        for (par, phi, o, f), r in zip(bj, refs):
            if r is None:
                continue
            scale = torch.maximum(o.abs(), r.abs()).amax(dim=0, keepdim=True)
            assert bool(((o - r).abs() <= 1e-12 * scale).all()), shape
        par, phi, o, f = bj[4]
        pick = np.array([0, 31, 32, 150, 299])
        J, env = oracle.jacobian_envelope(m, synth.CONV, phi.cpu().numpy()[:, pick], par.cpu().numpy()[pick])
        check_close(o.cpu().numpy()[:, pick], oracle.dense_to_csr_values(m, J), oracle.dense_to_csr_values(m, env),
                    RTOL_JAC, ATOL_JAC, f"{name} plan {shape}")


def test_graph_capture_replay_and_groups(pj, mechs):
    import torch
    m = mechs("h2co13")
    h = pj.pj_mech_create(m)
    sizes = [300, 5, 1200, 64, 900]
    bj = make_batches(torch, m, sizes, 60, synth.CONP, 1, h.nnz)
    refs = [pj.jacobian_sparse(h, synth.CONP, phi, par).clone() for (par, phi, _, _) in bj]
    st = torch.cuda.Stream()
    plan = pj.Plan(h, pj.PJ_OP_JACOBIAN, synth.CONP, bj, max_states_per_launch=1300)
    assert plan.config()["groups"] == 3
    with torch.cuda.stream(st):
        plan.capture(st)
        for _ in range(3):
            for (_, _, o, _) in bj:
                o.fill_(float("nan"))
            plan.launch(st)
    st.synchronize()
    for (_, _, o, _), r in zip(bj, refs):
        assert same_bits_but_rounding(o, r)
    # groups run one after another, so batches of different groups may share
    # output memory: two batches of two groups write the same buffer
    phi_a, par_a = synth.make_states(m, 400, 70, synth.CONP)
    phi_b, par_b = synth.make_states(m, 400, 71, synth.CONP)
    shared = torch.empty((h.nnz, 400), dtype=torch.float64, device="cuda")
    f = torch.empty((m.n_species + 1, 400), dtype=torch.float64, device="cuda")
    da = [torch.from_numpy(x).cuda() for x in (par_a, phi_a)]
    db = [torch.from_numpy(x).cuda() for x in (par_b, phi_b)]
    plan2 = pj.Plan(h, pj.PJ_OP_JACOBIAN, synth.CONP, [(da[0], da[1], shared, f), (db[0], db[1], shared, f)],
                    max_states_per_launch=400)
    plan2.run()
    torch.cuda.synchronize()
    assert same_bits_but_rounding(shared, pj.jacobian_sparse(h, synth.CONP, db[1], db[0]))


def test_autotune_and_cache(pj, mechs, tmp_path):
    import torch
    m = mechs("gri53")
    h = pj.pj_mech_create(m)
    bj = make_batches(torch, m, [2000, 513, 4096], 80, synth.CONP, 1, h.nnz)
    refs = [pj.jacobian_sparse(h, synth.CONP, phi, par).clone() for (par, phi, _, _) in bj]
    cache = str(tmp_path / "tune.jsonl")
    plan = pj.Plan(h, pj.PJ_OP_JACOBIAN, synth.CONP, bj)
    cfg = plan.autotune(cache_path=cache, reps=1)
    assert cfg["threads_per_block"] in (32, 64, 128, 256, 512) and 1 <= cfg["blocks_per_sm"] <= 16
    assert os.path.exists(cache) and "gri53" not in open(cache).read()  # keyed by hash, not name
    coop = cfg["threads_per_block"] >= 256

    def same(o, r, coop):
        return same_bits_but_rounding(o, r, 1e-12 if coop else 1e-13)
    plan.run()
    torch.cuda.synchronize()
    for (_, _, o, _), r in zip(bj, refs):
        assert same(o, r, coop)
    plan2 = pj.Plan(h, pj.PJ_OP_JACOBIAN, synth.CONP, bj)
    cfg2 = plan2.autotune(cache_path=cache, reps=1)
    assert cfg2 == cfg
    # every shape agrees with the entry point to rounding (the cooperative
    # shapes sum one entry from several warps)
    for shape in ((32, 1, 1), (64, 2, 0), (128, 4, 0), (512, 1, 1), (512, 1, 0), (256, 2, 1), (256, 1, 0)):
        plan2.set_config(*shape)
        plan2.run()
        torch.cuda.synchronize()
        for (_, _, o, _), r in zip(bj, refs):
            assert same(o, r, shape[0] >= 256), shape


@pytest.mark.parametrize("shape", [None, (128, 4, 0)])
def test_large_mechanism_plan_against_oracle_columns(pj, mechs, shape):
    """874 species / 3796 reactions: source terms and sampled Jacobian
    columns of a two-batch plan against the oracle, in the default shape
    (cooperative, per-state arrays in the workspace) and one state per
    thread."""
    import torch
    m = mechs("ic5874")
    h = pj.pj_mech_create(m)
    bj = make_batches(torch, m, [40, 3], 90, synth.CONP, 1, h.nnz)
    plan = pj.Plan(h, pj.PJ_OP_JACOBIAN, synth.CONP, bj)
    if shape is None:
        assert plan.config()["threads_per_block"] == 512 and plan.config()["use_shared"] == 0
    else:
        plan.set_config(*shape)
    plan.run()
    torch.cuda.synchronize()
    par, phi, o, f = bj[1]
    phi_h, par_h = phi.cpu().numpy(), par.cpu().numpy()
    ref, env = oracle.source_term_envelope(m, synth.CONP, phi_h, par_h)
    check_close(f.cpu().numpy(), ref, env, RTOL_SRC, ATOL_SRC, "874-species source terms")
    cols = [0, 1, 2, 300, 873]
    Jc = oracle.jacobian_columns(m, synth.CONP, phi_h, par_h, cols)
    rp, ci = h.sparsity(pj.PJ_CSR)
    vals = o.cpu().numpy()
    N1 = m.n_species + 1
    dense = np.zeros((N1, N1, phi_h.shape[1]))
    rows = np.repeat(np.arange(N1), np.diff(rp))
    dense[rows, ci] = vals
    got = dense[:, cols]
    scale = np.max(np.abs(Jc), axis=0, keepdims=True)
    assert np.all(np.abs(got - Jc) <= RTOL_JAC * np.abs(Jc) + 1e-12 * scale)
