"""Benchmark: Jacobian + source-term evaluations per second on GB300.

A step is one pass of the whole hot path over one batch: concentrations,
NASA-7 thermo, forward/reverse rate constants, pressure modification,
rates of progress, production rates, dT/dt and dV/dt, and the exact sparse
(CSR) Jacobian, all in one kernel launch (k_jacobian with source-term
output), for the 53-species / 325-reaction synthetic mechanism and 1,048,576
CONP states resident in HBM (inputs and outputs larger than L2).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank evaluates its own batch (replicas; weak
scaling) with no collective on the data path.
"""
from __future__ import annotations

import argparse
import tempfile
import json
import os
import statistics
import subprocess
import sys
import time

# the CPU oracle is timed on one core: keep numpy's BLAS single-threaded
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Jacobian & source-term evals/s (states/s) at FP64 tol vs oracle; roofline %"
UNIT = "states/s"
WORKLOAD = "gri53_1m"

# FP64 cost of an exp / log / divide in DFMA-equivalents: the kernels' exp is
# the table-driven one (9 FP64 operations: reduction 3, polynomial 4, table
# product 1, shift 1); log and divide are CUDA's, measured on this GB300 in
# DFMA issue slots (dfma 505 G/s, log 16.7 G/s, div 88.9 G/s).
W_EXP, W_LOG, W_DIV = 9.0, 30.2, 5.7
# FP64 peak derived from unit counts and clock: 2 DFMA / clock / SM
# (1.25 TFLOP/s nominal for GB300) x 152 SMs x 2070 MHz.
FP64_DFMA_PER_CLK_SM = 2.0


CPU_SAMPLE = 4096   # states of the oracle's timed sample (10-30 s of one core)


def fp64_work_per_state(m, jacobian=True):
    """Algorithmic FP64 work per state in DFMA-equivalents: every add, multiply
    and FMA of the formulas counts 1, exp 9 (the FP64 operations of the
    table-driven exp), log 30.2 and divide 5.7 (CUDA's routines on this part,
    in DFMA issue slots).
    The Jacobian's entry accumulations run as L2 reductions and are not
    counted."""
    import synth
    ns, nr = m.n_species, m.n_reactions
    w = 0.0
    w += (ns - 1) * W_DIV + (ns - 1) + 3 + W_DIV       # concentrations, C_tot, bath gas
    w += W_LOG + W_DIV + 15 * ns + ns                   # ln T, 1/T, NASA-7 cp/h/s/g, denominator
    for i in range(nr):
        r, p = m.reactants(i), m.products(i)
        nre, npr = len(r), len(p)
        sre, spr = sum(v for _, v in r), sum(v for _, v in p)
        kind = int(m.kind[i])
        w += 2 + W_EXP + (sre - 1) + 1                  # kf and forward product
        if kind == synth.PLOG:                          # segment search, two ln k, interpolation
            w += int(m.plog_ptr[i + 1] - m.plog_ptr[i]) + 2 * 2 + 3
        elif kind == synth.CHEB:                        # reduced T and P, recurrences, double sum
            nT, nP = (int(x) for x in m.cheb_shape[i])
            w += 4 + 2 * (nT + nP) + nT * nP + nT
        if m.reversible[i] and m.rev_explicit[i]:
            w += 2 + W_EXP + (spr - 1) + 1              # explicit reverse Arrhenius
        elif m.reversible[i]:
            w += (nre + npr) + 2 + W_EXP + (spr - 1) + 1
        if kind != synth.ELEMENTARY:
            w += len(m.efficiencies(i))
        if kind in (synth.LINDEMANN, synth.TROE, synth.SRI):
            w += 2 + W_EXP + 1 + W_DIV + 2             # k0/kinf, Pr, Pr/(1+Pr) F
            if kind == synth.TROE:
                w += (3 if m.troe_n[i] == 4 else 2) * W_EXP + 2 * W_LOG + W_EXP + W_DIV * 2 + 12
            elif kind == synth.SRI:
                w += 3 * W_EXP + 2 * W_LOG + W_DIV + 8
        w += 2 + (nre + npr)                            # q, production-rate scatter
        if jacobian:
            w += 2 + nre + (nre + npr)                  # dln kf/dT, dRf/dC, sum nu h
            if m.reversible[i]:
                w += 3 + npr
            if kind == synth.PLOG:
                w += 6
            elif kind == synth.CHEB:
                nT, nP = (int(x) for x in m.cheb_shape[i])
                w += 2 * (nT + nP) + nT * nP + nT + 2
            if kind == synth.THIRD_BODY:
                w += 4
            elif kind in (synth.LINDEMANN, synth.TROE, synth.SRI):
                w += 2 + 12 + W_DIV
                if kind == synth.TROE:
                    w += 16 + W_DIV
                elif kind == synth.SRI:
                    w += 10 + W_DIV
            w += 4 + (nre + npr) + 4 + 3 + 4          # dR/dT, dR/dS, dq/dT, dq/dS, dE, accumulators
            rows = sum(1 for k in range(ns - 1) if (sum(v for kk, v in p if kk == k) - sum(v for kk, v in r if kk == k)) != 0)
            slots = nre + (npr if m.reversible[i] else 0) + (len(m.efficiencies(i)) if kind != synth.ELEMENTARY else 0)
            w += 2 * rows + slots * (1 + rows + 2)     # products feeding the L2 reductions
    w += ns + 2 * (ns - 1) + W_DIV + 10                 # energy and state equations
    if jacobian:
        w += (ns + 1) * (12 + 2 * W_DIV) + 2 * ns + 4 * W_DIV   # T and S rows
    return w


def sample_clocks_start(path):
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                              "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=f, stderr=subprocess.DEVNULL)
        return p, f
    except Exception:
        return None, None


def sample_clocks_stop(handle, path, gpu_index):
    p, f = handle
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    f.close()
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or not parts[0].isdigit() or int(parts[0]) != gpu_index:
            continue
        try:
            sm.append(float(parts[1]))
            mx = float(parts[2])
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def oracle_baseline(m, mode, n_sample, seed):
    """The CPU oracle as it stands on a bounded sample (source terms + complex-step Jacobian)."""
    import oracle
    import synth
    phi, par = synth.make_states(m, n_sample, seed, mode)
    t0 = time.perf_counter()
    oracle.source_terms(m, mode, phi, par)
    J = oracle.jacobian(m, mode, phi, par)
    oracle.dense_to_csr_values(m, J)
    dt = time.perf_counter() - t0
    return n_sample / dt, dt


def _oracle_work(job):
    """One process's share of the parallel oracle timing."""
    import oracle
    m, mode, phi, par = job
    oracle.source_terms(m, mode, phi, par)
    oracle.dense_to_csr_values(m, oracle.jacobian(m, mode, phi, par))
    return phi.shape[1]


def _oracle_import(_):
    import oracle  # noqa: F401
    return 0


def oracle_baseline_parallel(m, mode, per_proc, seed, procs):
    """The same oracle on `procs` processes (spawned: the parent has used the
    GPU), per_proc states each; the pool is started and has imported the
    oracle before the clock starts."""
    import multiprocessing as mp
    import synth
    n = per_proc * procs
    phi, par = synth.make_states(m, n, seed, mode)
    jobs = [(m, mode, np.ascontiguousarray(phi[:, i * per_proc:(i + 1) * per_proc]),
             np.ascontiguousarray(par[i * per_proc:(i + 1) * per_proc])) for i in range(procs)]
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_import, range(procs), chunksize=1)
        t0 = time.perf_counter()
        done = sum(pool.map(_oracle_work, jobs, chunksize=1))
        dt = time.perf_counter() - t0
    return done / dt, dt


def _time(torch, stream, fn, reps=5):
    fn()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def lu_work_per_state(h):
    """FP64 work of one LU factorisation in DFMA-equivalents: for pivot k,
    |rows| x |cols| fused multiply-adds and |rows| multiplies, and one
    divide (rows/cols: the fill pattern's column below and row right of k)."""
    r, c = h.lu_pattern()
    N = h.n_species + 1
    rows = np.bincount(c[r > c], minlength=N)
    cols = np.bincount(r[c > r], minlength=N)
    return float(np.sum(rows * cols) + np.sum(rows) + N * W_DIV)


# ncu DRAM bytes per state of a kernel, recorded in profiles/ together with a
# hash of the kernel sources at capture time; a number is only used while
# the sources are unchanged.
PROFILE_OF = {("jac_csr", "gri53"): "k_jacobian_tm_gri53.md", ("source", "gri53"): "k_source_terms_gri53.md",
              ("lu", "gri53"): "k_lu_factor_gri53.md"}


def sources_hash():
    import hashlib
    d = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1809_01029_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".cpp", ".h")):
            d.update(f.encode())
            d.update(open(os.path.join(csrc, f), "rb").read())
    d.update(open(os.path.join(ROOT, "include", "pyjac_gb.h"), "rb").read())
    return d.hexdigest()[:16]


def kernel_traffic(op, mech_name):
    name = PROFILE_OF.get((op, mech_name))
    if not name:
        return None
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    import re
    m = re.search(r"traffic_bytes_per_state:\s*([0-9.eE+]+)\s+sources:\s*([0-9a-f]+)", open(path).read())
    if not m or m.group(2) != sources_hash():
        return None
    return float(m.group(1))


def lu_workloads(pj, synth, torch, dev, stream):
    """States/s of the Newton-matrix LU factorisation and solve: FP64 with
    M = I - h J formed from the FP64 Jacobian (53 species), and FP32 of the
    FP32 Newton matrix (111 species), 262,144 states each."""
    out = {}
    n = 262144
    for name, prec in (("gri53", pj.PJ_F64), ("usc111", pj.PJ_F32)):
        m = synth.make_mechanism(name)
        h = pj.pj_mech_create(m)
        N1 = m.n_species + 1
        phi_h, par_h = synth.make_states(m, n, 2018 + 3, synth.CONP)
        phi, par = torch.from_numpy(phi_h).to(dev), torch.from_numpy(par_h).to(dev)
        hs = torch.from_numpy(synth.make_step_sizes(n, 2018 + 3)).to(dev)
        f = torch.empty((N1, n), dtype=torch.float64, device=dev)
        lu_nnz, _ = h.lu_info()
        dt = torch.float64 if prec == pj.PJ_F64 else torch.float32
        vals = torch.empty((h.nnz, n), dtype=dt, device=dev)
        if prec == pj.PJ_F64:
            wb = h.workspace_size(pj.PJ_OP_JACOBIAN, n)
            w = torch.empty(max(wb, 1), dtype=torch.uint8, device=dev)
            pj.pj_eval_jacobian_sparse(h, synth.CONP, pj.PJ_CSR, n, par, phi, n, vals, f, None, w, wb, stream)
            hh = hs
        else:
            wb = h.workspace_size(pj.PJ_OP_NEWTON, n)
            w = torch.empty(max(wb, 1), dtype=torch.uint8, device=dev)
            pj.pj_newton_matrix_f32(h, synth.CONP, pj.PJ_CSR, n, par, phi, n, hs, 1.0, vals, f, None, w, wb, stream)
            hh = None
        del w
        lu = torch.empty((lu_nnz, n), dtype=dt, device=dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        wl = h.workspace_size(pj.PJ_OP_LU, n)
        w = torch.empty(max(wl, 1), dtype=torch.uint8, device=dev)
        reps = 3
        t = _time(torch, stream, lambda: pj.pj_lu_factor(h, prec, n, vals, n, lu, hh, 1.0, status, w, wl, stream),
                  reps=reps)
        tag = f"{name}_256k_lu_{'f64' if prec == pj.PJ_F64 else 'f32'}"
        out[f"{tag}_factor"] = n / (t * 1e-3)
        out[f"{tag}_states_flagged"] = int(status.item()) // (reps + 1)
        b = torch.randn((N1, n), dtype=dt, device=dev)
        x = torch.empty_like(b)
        t = _time(torch, stream, lambda: pj.pj_lu_solve(h, prec, n, lu, n, b, x, stream), reps=10)
        out[f"{tag}_solve"] = n / (t * 1e-3)
        del vals, lu, b, x, w, phi, par, hs, f
        torch.cuda.empty_cache()
    return out


def other_workloads(pj, synth, torch, dev, stream):
    """States/s of the other measured cases (one launch per evaluation)."""
    out = {}
    # 13 species / 27 reactions, 4096 states: source terms + CSR Jacobian
    m = synth.make_mechanism("h2co13")
    h = pj.pj_mech_create(m)
    n = 4096
    phi_h, par_h = synth.make_states(m, n, 2018 + 1, synth.CONP)
    phi, par = torch.from_numpy(phi_h).to(dev), torch.from_numpy(par_h).to(dev)
    v = torch.empty((h.nnz, n), dtype=torch.float64, device=dev)
    f = torch.empty((m.n_species + 1, n), dtype=torch.float64, device=dev)
    t = _time(torch, stream, lambda: pj.pj_eval_jacobian_sparse(h, synth.CONP, pj.PJ_CSR, n, par, phi, n, v, f,
                                                                None, None, 0, stream), reps=20)
    out["h2co13_4k_jacobian_csr"] = n / (t * 1e-3)
    # 111 species / 784 reactions, 262,144 states: FP32 Newton matrix vs FP64 Jacobian
    m = synth.make_mechanism("usc111")
    h = pj.pj_mech_create(m)
    n = 262144
    phi_h, par_h = synth.make_states(m, n, 2018 + 3, synth.CONP)
    phi, par = torch.from_numpy(phi_h).to(dev), torch.from_numpy(par_h).to(dev)
    hs = torch.from_numpy(synth.make_step_sizes(n, 2018 + 3)).to(dev)
    f = torch.empty((m.n_species + 1, n), dtype=torch.float64, device=dev)
    wb = h.workspace_size(pj.PJ_OP_NEWTON, n)
    w = torch.empty(max(wb, 1), dtype=torch.uint8, device=dev)
    M = torch.empty((h.nnz, n), dtype=torch.float32, device=dev)
    t = _time(torch, stream, lambda: pj.pj_newton_matrix_f32(h, synth.CONP, pj.PJ_CSR, n, par, phi, n, hs, 1.0, M, f,
                                                             None, w, wb, stream), reps=3)
    out["usc111_256k_newton_f32_csr"] = n / (t * 1e-3)
    del M
    J = torch.empty((h.nnz, n), dtype=torch.float64, device=dev)
    t = _time(torch, stream, lambda: pj.pj_eval_jacobian_sparse(h, synth.CONP, pj.PJ_CSR, n, par, phi, n, J, f, None,
                                                                w, wb, stream), reps=3)
    out["usc111_256k_jacobian_f64_csr"] = n / (t * 1e-3)
    del J, w
    # 53 species / 325 reactions, 65,536 states: adjoint VJP
    m = synth.make_mechanism("gri53")
    h = pj.pj_mech_create(m)
    n = 65536
    phi_h, par_h = synth.make_states(m, n, 2018 + 4, synth.CONP)
    phi, par = torch.from_numpy(phi_h).to(dev), torch.from_numpy(par_h).to(dev)
    uw_h, uT_h = synth.make_cotangents(m.n_species, n, 2018 + 4)
    uw, uT = torch.from_numpy(uw_h).to(dev), torch.from_numpy(uT_h).to(dev)
    y = torch.empty((m.n_species + 1, n), dtype=torch.float64, device=dev)
    g = torch.empty_like(y)
    gt = torch.empty((m.n_reactions, 3), dtype=torch.float64, device=dev)
    wb = h.workspace_size(pj.PJ_OP_VJP, n)
    w = torch.empty(max(wb, 1), dtype=torch.uint8, device=dev)
    t = _time(torch, stream, lambda: pj.pj_vjp(h, synth.CONP, n, par, phi, n, uw, uT, y, g, gt, None, w, wb, stream),
              reps=10)
    out["gri53_64k_vjp"] = n / (t * 1e-3)
    del y, g, gt, w, uw, uT
    # same states: analytical vs first-order finite-difference CSR Jacobian
    # (the paper's speedup comparison)
    f = torch.empty((m.n_species + 1, n), dtype=torch.float64, device=dev)
    J = torch.empty((h.nnz, n), dtype=torch.float64, device=dev)
    wb = h.workspace_size(pj.PJ_OP_JACOBIAN, n)
    w = torch.empty(max(wb, 1), dtype=torch.uint8, device=dev)
    ta = _time(torch, stream, lambda: pj.pj_eval_jacobian_sparse(h, synth.CONP, pj.PJ_CSR, n, par, phi, n, J, f,
                                                                 None, w, wb, stream), reps=10)
    wb = h.workspace_size(pj.PJ_OP_FD, n)
    w = torch.empty(max(wb, 1), dtype=torch.uint8, device=dev)
    tf = _time(torch, stream, lambda: pj.pj_eval_jacobian_fd(h, synth.CONP, pj.PJ_CSR, n, par, phi, n, J, f,
                                                             None, w, wb, stream), reps=2)
    out["gri53_64k_fd_jacobian_csr"] = n / (tf * 1e-3)
    out["gri53_64k_analytical_over_fd"] = tf / ta
    del J, f, w, phi, par
    torch.cuda.empty_cache()
    out.update(types_workload(pj, synth, torch, dev, stream))
    out.update(lu_workloads(pj, synth, torch, dev, stream))
    out.update(ragged_workload(pj, synth, torch, dev, stream))
    return out


def types_workload(pj, synth, torch, dev, stream):
    """The 53/325 mechanism with every less common reaction type (P-log,
    Chebyshev, chemically activated, explicit reverse), 1,048,576 states:
    source terms + CSR Jacobian, and its FP64-pipe fraction."""
    m = synth.make_mechanism("gri53_types")
    h = pj.pj_mech_create(m)
    n = 1048576
    phi_h, par_h = synth.make_states(m, n, 2018 + 2, synth.CONP)
    phi, par = torch.from_numpy(phi_h).to(dev), torch.from_numpy(par_h).to(dev)
    del phi_h, par_h
    f = torch.empty((m.n_species + 1, n), dtype=torch.float64, device=dev)
    wb = h.workspace_size(pj.PJ_OP_JACOBIAN, n)
    w = torch.empty(max(wb, 1), dtype=torch.uint8, device=dev)
    J = torch.empty((h.nnz, n), dtype=torch.float64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    t = _time(torch, stream, lambda: pj.pj_eval_jacobian_sparse(h, synth.CONP, pj.PJ_CSR, n, par, phi, n, J, f,
                                                                status, w, wb, stream), reps=3)
    ws = h.workspace_size(pj.PJ_OP_SOURCE, n)
    w2 = torch.empty(max(ws, 1), dtype=torch.uint8, device=dev)
    ts = _time(torch, stream, lambda: pj.pj_eval_source_terms(h, synth.CONP, n, par, phi, n, f, status, w2, ws,
                                                              stream), reps=5)
    assert int(status.item()) == 0
    props = torch.cuda.get_device_properties(dev)
    peak = FP64_DFMA_PER_CLK_SM * props.multi_processor_count * 2070.0e6
    out = {"gri53types_1m_jacobian_csr": n / (t * 1e-3),
           "gri53types_1m_jacobian_csr_fp64_frac": fp64_work_per_state(m) * n / (t * 1e-3) / peak,
           "gri53types_1m_source": n / (ts * 1e-3),
           "gri53types_1m_source_fp64_frac": fp64_work_per_state(m, jacobian=False) * n / (ts * 1e-3) / peak}
    del J, f, w, w2, phi, par
    torch.cuda.empty_cache()
    return out


def build_ragged(pj, synth, torch, dev, stream, scale=1.0, config=None, group_states=240000):
    """874 species / 3796 reactions, 32 log-uniform batches of 1,024..65,536
    states (each scaled by `scale`, at least 1): source terms + CSR Jacobian
    through one plan (persistent kernels, groups of <= group_states states
    sharing one output pool: three groups, 190 GB, whose 32-state tiles fill
    the resident warps' rounds better than five smaller groups), autotuned on
    the first six batches unless
    `config` (threads per block, blocks per SM, shared) is given, captured as
    a CUDA graph on its own stream."""
    m = synth.make_mechanism("ic5874")
    h = pj.pj_mech_create(m)
    sizes = [max(1, int(int(x) * scale)) for x in synth.ragged_batch_sizes()]
    N1 = m.n_species + 1
    # group assignment as the plan does it (consecutive batches)
    groups, cur, acc = [], [], 0
    for b, n in enumerate(sizes):
        if cur and acc + n > group_states:
            groups.append(cur)
            cur, acc = [], 0
        cur.append(b)
        acc += n
    groups.append(cur)
    pool_states = max(sum(sizes[b] for b in g) for g in groups)
    pool = torch.empty(pool_states * h.nnz, dtype=torch.float64, device=dev)
    fpool = torch.empty(pool_states * N1, dtype=torch.float64, device=dev)
    batches = []
    for g in groups:
        off = 0
        for b in g:
            n = sizes[b]
            phi_h, par_h = synth.make_states(m, n, 2018 + 5 + 7919 * b, synth.CONP)
            phi, par = torch.from_numpy(phi_h).to(dev), torch.from_numpy(par_h).to(dev)
            o = pool[off * h.nnz:(off + n) * h.nnz].view(h.nnz, n)
            f = fpool[off * N1:(off + n) * N1].view(N1, n)
            batches.append((par, phi, o, f))
            off += n
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    if config is None:
        cache = os.path.join(tempfile.gettempdir(), "pyjac_gb_autotune.jsonl")
        sample = pj.Plan(h, pj.PJ_OP_JACOBIAN, synth.CONP, batches[:6], status=status)
        cfg = sample.autotune(stream=stream, cache_path=cache, reps=1)
        del sample
        config = (cfg["threads_per_block"], cfg["blocks_per_sm"], cfg["use_shared"])
    plan = pj.Plan(h, pj.PJ_OP_JACOBIAN, synth.CONP, batches, max_states_per_launch=group_states, status=status)
    plan.set_config(*config)
    gs = torch.cuda.Stream(dev)
    plan.capture(gs)
    return {"m": m, "h": h, "plan": plan, "stream": gs, "status": status, "sizes": sizes, "groups": groups,
            "total": sum(sizes), "keep": (batches, pool, fpool)}


def ragged_workload(pj, synth, torch, dev, stream):
    """States/s of the 874-species ragged workload (see build_ragged), timed
    by graph replay."""
    r = build_ragged(pj, synth, torch, dev, stream)
    plan, gs = r["plan"], r["stream"]
    plan.launch(gs)
    gs.synchronize()
    t = _time(torch, gs, lambda: plan.launch(gs), reps=2)
    assert int(r["status"].item()) == 0
    total = r["total"]
    res = {"ic5874_ragged_jacobian_csr_graph": total / (t * 1e-3),
           "ic5874_ragged_info": {"batches": len(r["sizes"]), "states": total, "groups": len(r["groups"]),
                                  "config": plan.config(), "ms_per_replay": t}}
    del plan, r
    torch.cuda.empty_cache()
    return res


def run_reference(args, rank, world):
    import synth
    if rank != 0:
        return
    m = synth.make_mechanism("gri53")
    n_sample = 512
    times = []
    for _ in range(args.warmup):
        oracle_baseline(m, synth.CONP, 64, 7)
    for s in range(args.steps):
        _, dt = oracle_baseline(m, synth.CONP, n_sample, 2018 + 2 + s)
        times.append(dt)
    v = n_sample * args.steps / sum(times)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "mechanism": "synthetic 53 species / 325 reactions", "mode": "CONP",
                   "output": "source terms + CSR Jacobian", "sample_states_per_step": n_sample},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{n_sample} states per step of the {WORKLOAD} workload (numpy, complex-step Jacobian)"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def run_ragged(args, rank, world, local, torch, dist, synth, pj):
    """--op ragged: one step is one replay of the 874-species ragged plan
    (all 32 batches, or --n states in the same proportions)."""
    from paper_1809_01029_gb300 import replicas
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    scale = args.n / 623411.0 if args.n else 1.0
    cfg = tuple(int(x) for x in args.ragged_config.split(",")) if args.ragged_config else None
    r = build_ragged(pj, synth, torch, dev, stream, scale=scale, config=cfg)
    plan, gs, n, m = r["plan"], r["stream"], r["total"], r["m"]
    for _ in range(args.warmup):
        plan.launch(gs)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk_dir = args.clocks_dir or tempfile.gettempdir()
    os.makedirs(clk_dir, exist_ok=True)
    clk_path = os.path.join(clk_dir, f"bench_clocks_r{rank}.csv")
    clk = sample_clocks_start(clk_path)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(gs)
    for _ in range(args.steps):
        plan.launch(gs)
    e1.record(gs)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clocks = sample_clocks_stop(clk, clk_path, local)
    if world > 1:
        dist.barrier()
    ms_max = replicas.max_over_ranks(ms, dist if world > 1 else None)
    assert int(r["status"].item()) == 0, "invalid states in the benchmark batches"
    fp64_work = fp64_work_per_state(m)
    achieved = fp64_work * n / (ms * 1e-3) / 1e9
    props = torch.cuda.get_device_properties(dev)
    sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = FP64_DFMA_PER_CLK_SM * props.multi_processor_count * sm_max * 1e6 / 1e9
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G DFMA-equiv/s (FP64 pipe)",
                "frac": achieved / peak, "traffic": None, "kernel": "k_batched", "work_per_state": fp64_work,
                "peak_source": "derived: 2 FP64 FMA/clk/SM x SMs x max SM clock"}
    tr = kernel_traffic("ragged", "ic5874")
    if tr is not None:
        roofline["traffic"] = tr * n
        roofline["traffic_source"] = "ncu dram bytes per state of the current kernel sources x states"
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": n * world / (ms_max * 1e-3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "ic5874_ragged", "mechanism": "synthetic 874 species / 3796 reactions (seed %d)"
                       % synth.SPECS["ic5874"].seed, "states_per_gpu": n, "batches": len(r["sizes"]),
                       "groups": len(r["groups"]), "plan": plan.config(), "mode": "CONP", "op": "ragged",
                       "output": "source terms + CSR Jacobian (nnz %d) per batch, CUDA-graph replay" % r["h"].nnz,
                       "l2": "outputs larger than L2", "parallelism": f"replicas x{world}"},
            "roofline": roofline, "cpu_baseline": None, "e2e": None, "clocks": clocks,
            "gpu_launches": args.steps * len(r["groups"]), "variants": {}}))
    del plan, r
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=None, help="states per GPU (default: the workload's)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--clocks-dir", default=None, help="where to keep the nvidia-smi clock samples (default: a temp dir)")
    ap.add_argument("--op", default="jac_csr",
                    choices=["jac_csr", "jac_csc", "jac_dense", "source", "newton", "vjp", "lu", "ragged"],
                    help="what one step evaluates (default: source terms + CSR Jacobian)")
    ap.add_argument("--ragged-config", default=None,
                    help="ragged op: threads_per_block,blocks_per_sm,use_shared instead of autotuning")
    ap.add_argument("--mode", default="conp", choices=["conp", "conv"])
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    import synth
    import paper_1809_01029_gb300 as pj

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    pj.load_library()
    if args.op == "ragged":
        return run_ragged(args, rank, world, local, torch, dist, synth, pj)
    mech_name = {"newton": "usc111"}.get(args.op, "gri53")
    default_n = {"newton": 262144, "vjp": 65536, "lu": 262144}.get(args.op, 1048576)
    m = synth.make_mechanism(mech_name)
    h = pj.pj_mech_create(m)
    n = args.n or default_n
    mode = synth.CONP if args.mode == "conp" else synth.CONV
    phi_h, par_h = synth.make_states(m, n, 2018 + 2 + 1000 * rank, mode)
    dev = torch.device("cuda", local)
    phi = torch.from_numpy(phi_h).to(dev)
    par = torch.from_numpy(par_h).to(dev)
    N1 = m.n_species + 1
    if args.op == "newton":
        vals = torch.empty((h.nnz, n), dtype=torch.float32, device=dev)
        hstep = torch.from_numpy(synth.make_step_sizes(n, 2018 + 3)).to(dev)
    elif args.op == "vjp":
        uw_h, uT_h = synth.make_cotangents(m.n_species, n, 2018 + 4)
        u_w, u_T = torch.from_numpy(uw_h).to(dev), torch.from_numpy(uT_h).to(dev)
        vals = torch.empty((N1, n), dtype=torch.float64, device=dev)          # g_phi
        g_th = torch.empty((m.n_reactions, 3), dtype=torch.float64, device=dev)
    else:
        vals = torch.empty((N1 * N1 if args.op == "jac_dense" else h.nnz, n), dtype=torch.float64, device=dev)
    dphi = torch.empty((m.n_species + 1, n), dtype=torch.float64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    wb = h.workspace_size(pj.PJ_OP_JACOBIAN, n)
    work = torch.empty(max(wb, 1), dtype=torch.uint8, device=dev)
    wbs = h.workspace_size(pj.PJ_OP_SOURCE, n)
    work_s = torch.empty(max(wbs, 1), dtype=torch.uint8, device=dev)
    if args.op == "vjp":
        wb = h.workspace_size(pj.PJ_OP_VJP, n)
        work = torch.empty(max(wb, 1), dtype=torch.uint8, device=dev)
    if args.op == "lu":
        # factor M = I - h J formed from the FP64 CSR Jacobian of the states
        hstep = torch.from_numpy(synth.make_step_sizes(n, 2018 + 3)).to(dev)
        pj.pj_eval_jacobian_sparse(h, mode, pj.PJ_CSR, n, par, phi, n, vals, dphi, status, work, wb, stream)
        lu_nnz, _ = h.lu_info()
        lu = torch.empty((lu_nnz, n), dtype=torch.float64, device=dev)
        wb = h.workspace_size(pj.PJ_OP_LU, n)
        work = torch.empty(max(wb, 1), dtype=torch.uint8, device=dev)

    def step():
        if args.op == "source":
            pj.pj_eval_source_terms(h, mode, n, par, phi, n, dphi, status, work_s, wbs, stream)
        elif args.op == "newton":
            pj.pj_newton_matrix_f32(h, mode, pj.PJ_CSR, n, par, phi, n, hstep, 1.0, vals, dphi, status, work, wb,
                                    stream)
        elif args.op == "vjp":
            pj.pj_vjp(h, mode, n, par, phi, n, u_w, u_T, dphi, vals, g_th, status, work, wb, stream)
        elif args.op == "jac_dense":
            pj.pj_eval_jacobian_dense(h, mode, n, par, phi, n, vals, dphi, status, work, wb, stream)
        elif args.op == "lu":
            pj.pj_lu_factor(h, pj.PJ_F64, n, vals, n, lu, hstep, 1.0, status, work, wb, stream)
        else:
            fmt = pj.PJ_CSC if args.op == "jac_csc" else pj.PJ_CSR
            pj.pj_eval_jacobian_sparse(h, mode, fmt, n, par, phi, n, vals, dphi, status, work, wb, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk_dir = args.clocks_dir or tempfile.gettempdir()
    os.makedirs(clk_dir, exist_ok=True)
    clk_path = os.path.join(clk_dir, f"bench_clocks_r{rank}.csv")
    clk = sample_clocks_start(clk_path)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clocks = sample_clocks_stop(clk, clk_path, local)
    from paper_1809_01029_gb300 import replicas
    if world > 1:
        dist.barrier()
    ms_max = replicas.max_over_ranks(ms, dist if world > 1 else None)
    value = n * world / (ms_max * 1e-3)
    assert int(status.item()) == 0, "invalid states in the benchmark batch"

    # roofline of the (single) kernel of the step: FP64 pipe
    if args.op == "lu":
        fp64_work = lu_work_per_state(h)
    else:
        fp64_work = fp64_work_per_state(m, jacobian=args.op not in ("source",))
    achieved = fp64_work * n / (ms * 1e-3) / 1e9     # G DFMA-equivalent / s
    props = torch.cuda.get_device_properties(dev)
    sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = FP64_DFMA_PER_CLK_SM * props.multi_processor_count * sm_max * 1e6 / 1e9
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G DFMA-equiv/s (FP64 pipe)",
                "frac": achieved / peak, "traffic": None,
                "kernel": {"source": "k_source_terms", "vjp": "k_vjp", "lu": "k_lu_factor"}.get(args.op, "k_jacobian"),
                "work_per_state": fp64_work,
                "peak_source": "derived: 2 FP64 FMA/clk/SM x SMs x max SM clock"}
    tr = kernel_traffic(args.op, mech_name)
    if tr is not None:
        roofline["traffic"] = tr * n
        roofline["traffic_source"] = "ncu dram bytes per state of the current kernel sources x states"

    variants = {}
    if not args.no_variants and args.op == "jac_csr":
        def timeit(fn, reps=3):
            fn()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps
        # constant-volume cases on constant-volume states of the same recipe
        phv_h, pav_h = synth.make_states(m, n, 2018 + 2 + 1000 * rank, synth.CONV)
        phv, pav = torch.from_numpy(phv_h).to(dev), torch.from_numpy(pav_h).to(dev)
        del phv_h, pav_h
        for md, nm, ph_, pa_ in ((synth.CONP, "conp", phi, par), (synth.CONV, "conv", phv, pav)):
            t_src = timeit(lambda: pj.pj_eval_source_terms(h, md, n, pa_, ph_, n, dphi, status, work_s, wbs, stream))
            variants[f"source_{nm}"] = n / (t_src * 1e-3)
        variants["jacobian_csc_conp"] = n / (timeit(lambda: pj.pj_eval_jacobian_sparse(
            h, mode, pj.PJ_CSC, n, par, phi, n, vals, dphi, status, work, wb, stream)) * 1e-3)
        variants["jacobian_csr_conv"] = n / (timeit(lambda: pj.pj_eval_jacobian_sparse(
            h, synth.CONV, pj.PJ_CSR, n, pav, phv, n, vals, dphi, status, work, wb, stream)) * 1e-3)
        del phv, pav
        ha = h.with_jacobian_form(pj.PJ_JAC_APPROX)
        wba = ha.workspace_size(pj.PJ_OP_JACOBIAN, n)
        worka = torch.empty(max(wba, 1), dtype=torch.uint8, device=dev)
        variants["jacobian_csr_conp_approx"] = n / (timeit(lambda: pj.pj_eval_jacobian_sparse(
            ha, mode, pj.PJ_CSR, n, par, phi, n, vals, dphi, status, worka, wba, stream)) * 1e-3)
        variants["approx_nnz"] = ha.nnz
        del vals, worka
        torch.cuda.empty_cache()
        jd = torch.empty((N1 * N1, n), dtype=torch.float64, device=dev)
        variants["jacobian_dense_conp"] = n / (timeit(lambda: pj.pj_eval_jacobian_dense(
            h, mode, n, par, phi, n, jd, dphi, status, work, wb, stream)) * 1e-3)
        del jd
        torch.cuda.empty_cache()
        N1 = m.n_species + 1
    if args.op == "newton":
        vals = torch.empty((h.nnz, n), dtype=torch.float32, device=dev)
        hstep = torch.from_numpy(synth.make_step_sizes(n, 2018 + 3)).to(dev)
    elif args.op == "vjp":
        uw_h, uT_h = synth.make_cotangents(m.n_species, n, 2018 + 4)
        u_w, u_T = torch.from_numpy(uw_h).to(dev), torch.from_numpy(uT_h).to(dev)
        vals = torch.empty((N1, n), dtype=torch.float64, device=dev)          # g_phi
        g_th = torch.empty((m.n_reactions, 3), dtype=torch.float64, device=dev)
    else:
        vals = torch.empty((N1 * N1 if args.op == "jac_dense" else h.nnz, n), dtype=torch.float64, device=dev)

    if not args.no_variants and args.op == "jac_csr":
        variants.update(other_workloads(pj, synth, torch, dev, stream))

    e2e = None
    if not args.no_e2e and args.op == "jac_csr":
        # the same step through the C ABI with HOST buffers
        # (pj_eval_jacobian_sparse_host): page-locked states in, Jacobian
        # values and source terms out, the transfers inside the call, chunked
        # and overlapped with the kernels
        phi_pin = torch.from_numpy(phi_h).pin_memory()
        par_pin = torch.from_numpy(par_h).pin_memory()
        vals_pin = torch.empty((h.nnz, n), dtype=torch.float64).pin_memory()
        dphi_pin = torch.empty((m.n_species + 1, n), dtype=torch.float64).pin_memory()

        def e2e_step():
            bad = pj.pj_eval_jacobian_sparse_host(h, mode, pj.PJ_CSR, n, par_pin, phi_pin, vals_pin, dphi_pin,
                                                  0, stream)
            assert bad == 0
        e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        k = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        for _ in range(k):
            e2e_step()
        torch.cuda.synchronize()
        ms_e2e = replicas.max_over_ranks((time.perf_counter() - t0) * 1e3 / k, dist if world > 1 else None)

        # for comparison: the copies and the kernel one after another
        def serial_step():
            phi.copy_(phi_pin, non_blocking=True)
            par.copy_(par_pin, non_blocking=True)
            step()
            vals_pin.copy_(vals, non_blocking=True)
            dphi_pin.copy_(dphi, non_blocking=True)
        serial_step()
        torch.cuda.synchronize()
        ea = torch.cuda.Event(enable_timing=True)
        eb = torch.cuda.Event(enable_timing=True)
        ea.record(stream)
        serial_step()
        eb.record(stream)
        torch.cuda.synchronize()
        variants["e2e_serial_copies"] = n / (ea.elapsed_time(eb) * 1e-3)
        e2e = {"value": n * world / (ms_e2e * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(phi_pin.numel() * 8 + par_pin.numel() * 8),
               "d2h_bytes_per_step": int(vals_pin.numel() * 8 + dphi_pin.numel() * 8),
               "api": "pj_eval_jacobian_sparse_host (page-locked host buffers, host wall clock)"}
        del phi_pin, par_pin, vals_pin, dphi_pin

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu:
        n_cpu = CPU_SAMPLE if mech_name == "gri53" else CPU_SAMPLE // 4
        v, dt = oracle_baseline(m, mode, n_cpu, 2018 + 2)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n_cpu} states of the {m.name} mechanism: numpy source terms + complex-step CSR Jacobian "
                         f"({dt:.1f} s)"}
        if args.op == "jac_csr":
            procs = max(1, min(os.cpu_count() or 1, 64))
            try:
                va, dta = oracle_baseline_parallel(m, mode, CPU_SAMPLE, 2018 + 2, procs)
                cpu_all = {"value": va, "unit": UNIT, "cores": procs, "kind": "oracle",
                           "sample": f"{CPU_SAMPLE * procs} states of the {m.name} mechanism on {procs} processes "
                                     f"({dta:.1f} s)"}
            except Exception as e:  # noqa: BLE001 -- the figure is context only
                cpu_all = {"unavailable": str(e)[:200]}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": {"newton": "usc111_256k", "vjp": "gri53_vjp64k", "lu": "gri53_lu256k"}.get(args.op, WORKLOAD),
                   "mechanism": "synthetic %d species / %d reactions (seed %d)" % (
                       m.n_species, m.n_reactions, synth.SPECS[mech_name].seed),
                       "states_per_gpu": n, "mode": args.mode.upper(), "op": args.op,
                       "output": {"newton": "FP32 Newton matrix I - h J (CSR, nnz %d) + FP64 source terms" % h.nnz,
                                  "vjp": "y = (wdot, dT/dt), g_phi and summed g_theta",
                                  "jac_csr": "source terms + CSR Jacobian (nnz %d)" % h.nnz,
                                  "jac_csc": "source terms + CSC Jacobian (nnz %d)" % h.nnz,
                                  "jac_dense": "source terms + dense Jacobian (%d entries)" % (N1 * N1),
                                  "lu": "FP64 LU factors of I - h J (%d values)" % h.lu_info()[0],
                                  "source": "source terms"}[args.op],
                       "l2": "inputs and outputs larger than L2 (%.1f GB per step)" % ((h.nnz + 2 * (m.n_species + 1)) * n * 8 / 1e9),
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": args.steps * (2 if args.op == "vjp" else 1), "variants": variants}))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
