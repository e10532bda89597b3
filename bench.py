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

# FP64 peak derived from unit counts and clock: 2 DFMA / clock / SM
# (1.25 TFLOP/s nominal for GB300) x 152 SMs x 2070 MHz.
FP64_DFMA_PER_CLK_SM = 2.0
# FP32 FMA issue rate relative to FP64 on this part (128 vs 2 per clock per SM)
FP32_PER_FP64 = 64.0


CPU_SAMPLE = 4096   # states of the oracle's timed sample (10-30 s of one core)

# Algorithmic work per state: the operation counts of the oracle's formulas
# (a counting scalar run through the source terms, and forward-mode through
# their derivatives, by oracle/opcount.py), stored with their weights in
# oracle/work_counts.json by `python -m oracle.opcount` (the timed legs read
# the table and run no oracle code).
WORK_TABLE = os.path.join(ROOT, "oracle", "work_counts.json")
_WORK = None


def work_table():
    global _WORK
    if _WORK is None:
        with open(WORK_TABLE) as f:
            _WORK = json.load(f)
    return _WORK


def dfma_equiv(counts, weights):
    """FP64 work in DFMA-equivalents; entry accumulations ("acc") are L2
    reductions in the kernels, off the FP64 pipe, and are not counted."""
    return sum(weights[c] * counts[c] for c in counts if c != "acc")


def work_per_state(mech_name, op, mode="conp"):
    """(DFMA-equivalent FP64 work per state, the counts) of one evaluation:
    source terms; the Jacobian (source terms and forward-mode derivatives);
    the FP32 Newton matrix (the derivative part in FP32, at 1/64 of an FP64
    operation); the VJP (the derivatives of y, as the Jacobian's); the LU
    factorisation of the Newton matrix ("lu"), and with M = I - h gamma J
    formed from the Jacobian's values first ("newton_lu", what the factor
    kernel does when given J and h)."""
    t = work_table()
    w, c = t["weights"], t["counts"][mech_name]
    if op == "source":
        k = c[f"source_{mode}"]
        return dfma_equiv(k, w), k
    if op in ("lu", "newton_lu"):
        return dfma_equiv(c[op], w), c[op]
    k = c[f"jacobian_{mode}"]
    full = dfma_equiv(k, w)
    if op == "newton":
        src = dfma_equiv(c[f"source_{mode}"], w)
        return src + (full - src) / FP32_PER_FP64, k
    return full, k


def hbm_peak_gbs():
    """Measured copy bandwidth of the GB300s (MEASURED_PEAKS.json),
    else the fallback measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def algorithmic_bytes(op, ns, h):
    """Bytes one state's evaluation must move to or from HBM (8-byte values;
    the mechanism's constants are shared by all states and not counted):
    state Phi (Ns+1) and parameter in, outputs out."""
    N = ns + 1
    io = (N + 1) * 8
    if op == "source":
        return io + N * 8
    if op in ("jac_csr", "jac_csc"):
        return io + (h.nnz + N) * 8
    if op == "jac_dense":
        return io + (N * N + N) * 8
    if op == "newton":
        return io + 8 + h.nnz * 4 + N * 8
    if op == "vjp":
        return io + N * 8 + 2 * N * 8           # cotangents in; y and g_Phi out
    if op == "lu":
        return h.nnz * 8 + 8 + h.lu_info()[0] * 8
    return None


def t_roof(work, nbytes, n, ms, peak_g, weights):
    """The roofline time of the step, t_roof = max(bytes / HBM peak, sum over
    operation classes of ops_c / peak_c), each class's peak the FP64 pipe's
    DFMA rate divided by its cost in DFMA issue slots, and the fraction
    t_roof / t_measured."""
    hbm, src = hbm_peak_gbs()
    t_hbm = nbytes * n / (hbm * 1e9) * 1e3 if nbytes else 0.0
    t_fp64 = work * n / (peak_g * 1e9) * 1e3
    tr = max(t_hbm, t_fp64)
    return {"ms": tr, "frac": tr / ms, "hbm_ms": t_hbm, "fp64_ms": t_fp64, "bytes_per_state": nbytes,
            "hbm_gbs": hbm, "hbm_source": src,
            "class_peaks_g_per_s": {c: peak_g / weights[c] for c in weights if c != "acc"}}


def class_shares(counts, weights):
    """Share of each operation class in the FP64-pipe time of the count."""
    tot = dfma_equiv(counts, weights)
    return {cls: weights[cls] * v / tot for cls, v in counts.items() if cls != "acc" and v}


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


# The other workloads' oracle timing (--cpu-configs): each on a bounded
# sample, one core and every core.  (mechanism, what, states per process,
# Jacobian columns timed: None = all)
CPU_CONFIGS = [("h2co13", "source + CSR Jacobian", 2048, None),
               ("gri53", "source + CSR Jacobian", 512, None),
               ("usc111", "source + FP64 Newton matrix", 64, None),
               ("gri53", "VJP", 256, None),
               ("ic5874", "source + CSR Jacobian", 4, 16)]


def _oracle_config_work(job):
    """One process's share of a configuration's oracle timing: the seconds
    for its states (for the 874-species Jacobian, `cols` of the 875 columns
    timed and the time scaled to all of them)."""
    import oracle
    m, what, phi, par, cols = job
    t0 = time.perf_counter()
    if what == "VJP":
        import synth
        uw, uT = synth.make_cotangents(m.n_species, phi.shape[1], 5)
        oracle.vjp(m, 0, phi, par, uw, uT)
    else:
        oracle.source_terms(m, 0, phi, par)
        if cols is None:
            J = oracle.jacobian(m, 0, phi, par)
            if what.endswith("Newton matrix"):
                N1 = m.n_species + 1
                J = -1e-7 * J
                J[np.arange(N1), np.arange(N1)] += 1.0
            oracle.dense_to_csr_values(m, J)
        else:
            t1 = time.perf_counter()
            oracle.jacobian_columns(m, 0, phi, par, list(range(cols)))
            return (t1 - t0) + (time.perf_counter() - t1) * (m.n_species + 1) / cols
    return time.perf_counter() - t0


def cpu_baseline_configs(procs):
    """States/s of the oracle on every configuration's workload, on one core
    and on `procs` spawned processes (bounded samples)."""
    import multiprocessing as mp
    import synth
    out = []
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_import, range(procs), chunksize=1)
        for name, what, per, cols in CPU_CONFIGS:
            m = synth.make_mechanism(name)
            phi, par = synth.make_states(m, per * procs, 2018 + 9, synth.CONP)
            dt1 = _oracle_config_work((m, what, phi[:, :per], par[:per], cols))
            jobs = [(m, what, np.ascontiguousarray(phi[:, i * per:(i + 1) * per]),
                     np.ascontiguousarray(par[i * per:(i + 1) * per]), cols) for i in range(procs)]
            t0 = time.perf_counter()
            secs = pool.map(_oracle_config_work, jobs, chunksize=1)
            dta = time.perf_counter() - t0 if cols is None else max(secs)
            out.append({"mechanism": name, "what": what, "one_core_states_per_s": per / dt1,
                        "all_cores_states_per_s": per * procs / dta, "cores": procs,
                        "sample_states_per_process": per,
                        "note": None if cols is None else f"Jacobian time scaled from {cols} of the "
                                                          f"{m.n_species + 1} columns"})
    return out


def batch_sweep(pj, synth, torch, dev, stream):
    """States/s against batch size (the GB300 counterpart of Sec. 3.5.1's
    GPU saturation study): source terms and source terms + CSR Jacobian of
    the 53/325 mechanism, one launch each, 1 ki .. 1 Mi states."""
    m = synth.make_mechanism("gri53")
    h = pj.pj_mech_create(m)
    N1 = m.n_species + 1
    nmax = 1 << 20
    phi_h, par_h = synth.make_states(m, nmax, 2018 + 2, synth.CONP)
    phi, par = torch.from_numpy(phi_h).to(dev), torch.from_numpy(par_h).to(dev)
    del phi_h, par_h
    f = torch.empty((N1, nmax), dtype=torch.float64, device=dev)
    J = torch.empty((h.nnz, nmax), dtype=torch.float64, device=dev)
    out = {}
    for lg in range(10, 21, 2):
        n = 1 << lg
        ws = h.workspace_size(pj.PJ_OP_SOURCE, n)
        w = torch.empty(max(ws, 1), dtype=torch.uint8, device=dev)
        reps = max(3, min(200, (1 << 22) // n))
        ts = _time(torch, stream, lambda: pj.pj_eval_source_terms(h, synth.CONP, n, par, phi, nmax, f, None, w, ws,
                                                                  stream), reps=reps)
        wj = h.workspace_size(pj.PJ_OP_JACOBIAN, n)
        w2 = torch.empty(max(wj, 1), dtype=torch.uint8, device=dev)
        tj = _time(torch, stream, lambda: pj.pj_eval_jacobian_sparse(h, synth.CONP, pj.PJ_CSR, n, par, phi, nmax, J,
                                                                     f, None, w2, wj, stream),
                   reps=max(3, reps // 3))
        out[str(n)] = {"source": n / (ts * 1e-3), "jacobian_csr": n / (tj * 1e-3)}
    del J, f, phi, par
    torch.cuda.empty_cache()
    return out


def fp64_peak(torch, dev, sm_mhz=2070.0):
    """Derived FP64 peak, DFMA per second: 2 per clock per SM x SMs x clock."""
    return FP64_DFMA_PER_CLK_SM * torch.cuda.get_device_properties(dev).multi_processor_count * sm_mhz * 1e6


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


# Per-state ncu figures of a kernel (DRAM bytes, executed FP64-pipe
# instructions), recorded in profiles/ together with a hash of the kernel
# sources at capture time; a number is only used while the sources are
# unchanged.
PROFILE_OF = {("k_jacobian_coop", "gri53"): "k_jacobian_coop_gri53.md",
              ("k_jacobian_tm", "gri53"): "k_jacobian_tm_gri53.md",
              ("k_source_terms", "gri53"): "k_source_terms_gri53.md",
              ("k_lu_factor_v", "gri53"): "k_lu_factor_gri53.md",
              ("k_jacobian_coop", "usc111"): "k_jacobian_coop_usc111.md",
              ("k_jacobian_coop", "ic5874"): "k_jacobian_coop_ic5874.md"}


def sources_hash():
    """Hash of the kernel sources (paper_1809_01029_gb300/csrc and the C
    header) with comments and blank lines removed, so that a profile's
    figures stay attached to the code they measured across comment edits."""
    import hashlib
    import re
    d = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1809_01029_gb300", "csrc")
    files = [os.path.join(csrc, f) for f in sorted(os.listdir(csrc)) if f.endswith((".cu", ".cuh", ".cpp", ".h"))]
    files.append(os.path.join(ROOT, "include", "pyjac_gb.h"))
    for path in files:
        text = open(path, encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        d.update(os.path.basename(path).encode())
        d.update(code.encode())
    return d.hexdigest()[:16]


def _profile_figure(kern, mech_name, key):
    name = PROFILE_OF.get((kern, mech_name))
    if not name:
        return None
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    import re
    m = re.search(key + r":\s*([0-9.eE+]+)\s+sources:\s*([0-9a-f]+)", open(path).read())
    if not m or m.group(2) != sources_hash():
        return None
    return float(m.group(1))


def kernel_traffic(op, mech_name, kern):
    """DRAM bytes per state of the kernel's profile (None once stale)."""
    return _profile_figure(kern, mech_name, "traffic_bytes_per_state")


def kernel_executed(op, mech_name, kern):
    """Executed FP64-pipe instructions per state of the kernel's profile."""
    return _profile_figure(kern, mech_name, "fp64_pipe_instr_per_state")


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
        if prec == pj.PJ_F64:
            out[f"{tag}_factor_fp64_frac"] = (work_per_state(name, "newton_lu")[0] * n / (t * 1e-3) /
                                              fp64_peak(torch, dev))
        out[f"{tag}_states_flagged"] = int(status.item()) // (reps + 1)
        if prec == pj.PJ_F32:
            out[f"{tag}_flagged_states"] = lu_nonfinite_states(torch, h, vals, lu, hs)
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
    peak = fp64_peak(torch, dev)
    out["usc111_256k_newton_f32_csr_fp64_frac"] = work_per_state("usc111", "newton")[0] * n / (t * 1e-3) / peak
    J = torch.empty((h.nnz, n), dtype=torch.float64, device=dev)
    t = _time(torch, stream, lambda: pj.pj_eval_jacobian_sparse(h, synth.CONP, pj.PJ_CSR, n, par, phi, n, J, f, None,
                                                                w, wb, stream), reps=3)
    out["usc111_256k_jacobian_f64_csr"] = n / (t * 1e-3)
    out["usc111_256k_jacobian_f64_csr_fp64_frac"] = work_per_state("usc111", "jacobian")[0] * n / (t * 1e-3) / peak
    out["usc111_256k_newton_f32_error"] = newton_f32_error(torch, h, M, J, hs)
    del M, J, w
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
    out["gri53_64k_vjp_fp64_frac"] = work_per_state("gri53", "vjp")[0] * n / (t * 1e-3) / peak
    del y, g, gt, w, uw, uT
    # same states: analytical vs first-order finite-difference CSR Jacobian
    # (the paper's speedup comparison)
    f = torch.empty((m.n_species + 1, n), dtype=torch.float64, device=dev)
    J = torch.empty((h.nnz, n), dtype=torch.float64, device=dev)
    wb = h.workspace_size(pj.PJ_OP_JACOBIAN, n)
    w = torch.empty(max(wb, 1), dtype=torch.uint8, device=dev)
    ta = _time(torch, stream, lambda: pj.pj_eval_jacobian_sparse(h, synth.CONP, pj.PJ_CSR, n, par, phi, n, J, f,
                                                                 None, w, wb, stream), reps=10)
    out["gri53_64k_jacobian_csr"] = n / (ta * 1e-3)
    tn = _time(torch, stream, lambda: pj.pj_eval_jacobian_sparse_noalloc(h, synth.CONP, pj.PJ_CSR, n, par, phi, n, J,
                                                                         f, None, stream), reps=10)
    out["gri53_64k_jacobian_csr_noalloc"] = n / (tn * 1e-3)
    wb = h.workspace_size(pj.PJ_OP_FD, n)
    w = torch.empty(max(wb, 1), dtype=torch.uint8, device=dev)
    tf = _time(torch, stream, lambda: pj.pj_eval_jacobian_fd(h, synth.CONP, pj.PJ_CSR, n, par, phi, n, J, f,
                                                             None, w, wb, stream), reps=2)
    out["gri53_64k_fd_jacobian_csr"] = n / (tf * 1e-3)
    out["gri53_64k_analytical_over_fd"] = tf / ta
    del J, f, w, phi, par
    torch.cuda.empty_cache()
    out["gri53_batch_sweep"] = batch_sweep(pj, synth, torch, dev, stream)
    out.update(types_workload(pj, synth, torch, dev, stream))
    out.update(lu_workloads(pj, synth, torch, dev, stream))
    out.update(ragged_workload(pj, synth, torch, dev, stream))
    return out


def newton_f32_error(torch, h, M, J, hs, gamma=1.0, chunk=16384):
    """Error of the FP32 Newton matrix M against M64 = I - h gamma J formed
    in FP64 from the FP64 Jacobian of the same states (itself held to the
    oracle by the parity tests), over every state of the batch: per state
    ||M - M64||_F / ||M64||_F, and per entry |M - M64| / max_ij |M64| of
    its state; plus how many states have a non-finite FP32 entry."""
    ptr, idx = h.sparsity()
    rows = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr))
    diag = torch.from_numpy(np.nonzero(rows == idx)[0]).to(M.device)
    n = M.shape[1]
    frob, ent, nonfinite = [], [], 0
    for s0 in range(0, n, chunk):
        s1 = min(n, s0 + chunk)
        M64 = -(gamma * hs[s0:s1])[None, :] * J[:, s0:s1]
        M64[diag] += 1.0
        d = M[:, s0:s1].double() - M64
        ok = torch.isfinite(d).all(0)
        nonfinite += int((~ok).sum())
        d, M64 = d[:, ok], M64[:, ok]
        frob.append(torch.linalg.vector_norm(d, dim=0) / torch.linalg.vector_norm(M64, dim=0))
        ent.append(d.abs().amax(0) / M64.abs().amax(0))
    frob, ent = torch.cat(frob), torch.cat(ent)
    q = lambda x, p: float(torch.quantile(x.float().cpu(), p))
    return {"against": "M64 = I - h gamma J from the FP64 Jacobian of the same states, every state",
            "frobenius_rel": {"median": q(frob, 0.5), "p99": q(frob, 0.99), "max": float(frob.max())},
            "max_entry_rel_to_state_max": {"median": q(ent, 0.5), "p99": q(ent, 0.99), "max": float(ent.max())},
            "nonfinite_states": nonfinite}


def lu_nonfinite_states(torch, h, vals, lu, hs):
    """Which states the FP32 LU flags, and where: how many; the median of
    max |M| over flagged and over finite states; the pivot step (min(row,
    col) of the first non-finite factor value in storage order) histogram;
    and how many flagged states had a non-finite M to begin with."""
    bad = ~torch.isfinite(lu).all(0)
    k = int(bad.sum())
    if k == 0:
        return {"states": 0}
    amax = vals.abs().amax(0).double()
    Mbad = ~torch.isfinite(vals).all(0)
    rows, cols = h.lu_pattern()
    piv = torch.from_numpy(np.minimum(rows, cols)).to(lu.device)
    first = (~torch.isfinite(lu[:, bad])).int().argmax(0)
    steps, counts = torch.unique(piv[first], return_counts=True)
    order = torch.argsort(counts, descending=True)[:8]
    return {"states": k, "of": int(lu.shape[1]), "with_nonfinite_M": int((Mbad & bad).sum()),
            "max_abs_M_median_flagged": float(amax[bad & ~Mbad].median()) if int((bad & ~Mbad).sum()) else None,
            "max_abs_M_median_finite": float(amax[~bad].median()),
            "h_median_flagged": float(hs[bad].median()), "h_median_finite": float(hs[~bad].median()),
            "first_nonfinite_pivot_step": {int(steps[i]): int(counts[i]) for i in order}}


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
    peak = fp64_peak(torch, dev)
    out = {"gri53types_1m_jacobian_csr": n / (t * 1e-3),
           "gri53types_1m_jacobian_csr_fp64_frac": work_per_state("gri53_types", "jacobian")[0] * n / (t * 1e-3) / peak,
           "gri53types_1m_source": n / (ts * 1e-3),
           "gri53types_1m_source_fp64_frac": work_per_state("gri53_types", "source")[0] * n / (ts * 1e-3) / peak}
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


def plan_kernel(plan):
    """The kernel a batched plan's launch shape runs: 256 or 512 threads per
    block are the cooperative layout."""
    return "k_jacobian_coop" if plan.config()["threads_per_block"] >= 256 else "k_batched"


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
           "ic5874_ragged_jacobian_csr_graph_fp64_frac":
               work_per_state("ic5874", "jacobian")[0] * total / (t * 1e-3) / fp64_peak(torch, dev),
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
    fp64_work, counts = work_per_state("ic5874", "jacobian")
    achieved = fp64_work * n / (ms * 1e-3) / 1e9
    props = torch.cuda.get_device_properties(dev)
    sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = FP64_DFMA_PER_CLK_SM * props.multi_processor_count * sm_max * 1e6 / 1e9
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G DFMA-equiv/s (FP64 pipe)",
                "frac": achieved / peak, "traffic": None, "kernel": plan_kernel(plan), "work_per_state": fp64_work,
                "work_source": "oracle operation count (oracle/work_counts.json)", "counts": counts,
                "peak_source": "derived: 2 FP64 FMA/clk/SM x SMs x max SM clock"}
    tr = kernel_traffic("ragged", "ic5874", plan_kernel(plan))
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
    ap.add_argument("--cpu-configs", action="store_true",
                    help="also time the oracle on every configuration's workload (bounded samples, one and all cores)")
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

    # roofline of the (single) kernel of the step: FP64 pipe, against the
    # method's operation count (oracle table) and, beside it, the FP64-pipe
    # instructions the kernel executed (ncu, recorded in profiles/)
    wop = {"jac_csr": "jacobian", "jac_csc": "jacobian", "jac_dense": "jacobian", "lu": "newton_lu"}.get(args.op,
                                                                                                        args.op)
    fp64_work, counts = work_per_state(mech_name, wop, args.mode)
    achieved = fp64_work * n / (ms * 1e-3) / 1e9     # G DFMA-equivalent / s
    sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = fp64_peak(torch, dev, sm_max) / 1e9
    weights = work_table()["weights"]
    kern = {"source": "k_source_terms", "vjp": "k_vjp", "lu": "k_lu_factor_v"}.get(args.op) or \
        {0: "k_jacobian", 1: "k_jacobian_tm", 2: "k_jacobian_coop"}[h.jacobian_layout(
            pj.PJ_DENSE if args.op == "jac_dense" else pj.PJ_CSR, pj.PJ_F32 if args.op == "newton" else pj.PJ_F64, n)]
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G DFMA-equiv/s (FP64 pipe)",
                "frac": achieved / peak, "traffic": None, "kernel": kern,
                "work_per_state": fp64_work,
                "work_source": "oracle operation count (oracle/work_counts.json, oracle/opcount.py): add, mul, "
                               "fma 1, exp 9, log 30.2, div 5.7 DFMA-equivalents; entry accumulations (L2 "
                               "reductions) not counted",
                "counts": counts, "class_shares": class_shares(counts, weights),
                "peak_source": "derived: 2 FP64 FMA/clk/SM x SMs x max SM clock"}
    roofline["t_roof"] = t_roof(fp64_work, algorithmic_bytes(args.op, m.n_species, h), n, ms, peak, weights)
    ex = kernel_executed(args.op, mech_name, kern)
    if ex is not None:
        roofline["executed"] = {"fp64_pipe_instr_per_state": ex, "frac": ex * n / (ms * 1e-3) / 1e9 / peak,
                                "source": "ncu sm__inst_executed_pipe_fp64 x 32 per state of the current sources"}
    tr = kernel_traffic(args.op, mech_name, kern)
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
        # the low-DRAM-traffic shape of the cooperative kernel (16 warps x 1
        # block per SM; the library reads the layout variables at launch)
        lay_env = {"PYJAC_GB_JAC_LAYOUT": "coop", "PYJAC_GB_COOP_WARPS": "16", "PYJAC_GB_COOP_CTAS": "1"}
        saved = {k: os.environ.get(k) for k in lay_env}
        os.environ.update(lay_env)
        variants["jacobian_csr_conp_coop16x1"] = n / (timeit(lambda: pj.pj_eval_jacobian_sparse(
            h, mode, pj.PJ_CSR, n, par, phi, n, vals, dphi, status, work, wb, stream)) * 1e-3)
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
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
        if args.cpu_configs:
            variants["cpu_baseline_configs"] = cpu_baseline_configs(max(1, min(os.cpu_count() or 1, 64)))

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
