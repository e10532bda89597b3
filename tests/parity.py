"""Comparison helpers for GPU-vs-oracle parity tests.

Floating-point bar (stated in the benchmark spec's tolerances and derived in the
design notes): |gpu - ref| <= rtol * max(|ref|, env) + atol, where env is the
oracle's absolute envelope (the sum of magnitudes of the terms that make up
the value; near chemical equilibrium net rates are differences of nearly
equal forward and reverse rates, Sec. 3.2).  rtol = 1e-10, atol = 1e-20 for
source terms; rtol = 1e-8 per Jacobian entry.
"""
import numpy as np

RTOL_SRC, ATOL_SRC = 1e-10, 1e-20
RTOL_JAC, ATOL_JAC = 1e-8, 1e-20


def check_close(got, ref, env, rtol, atol, what=""):
    got = np.asarray(got)
    ref = np.asarray(ref)
    env = np.maximum(np.asarray(env), np.abs(ref))
    err = np.abs(got - ref)
    tol = rtol * env + atol
    bad = ~(err <= tol)
    if bad.any():
        idx = np.unravel_index(np.argmax(np.where(bad, err / np.maximum(tol, 1e-300), 0)), err.shape)
        raise AssertionError(
            f"{what}: {bad.sum()} / {bad.size} entries out of tolerance; worst at {idx}: "
            f"gpu={got[idx]!r} ref={ref[idx]!r} env={env[idx]!r} err={err[idx]!r} tol={tol[idx]!r}")
    needed_env = int(np.sum(err > rtol * np.abs(ref) + atol))
    return needed_env


def paper_error_norms(J_gpu, J_ref, C_thresh=1e20):
    """The paper's LAPACK-style norm E_L and filtered norm E_C (Sec. 3.3,
    Jacobian verification) over states on the last axis."""
    J_gpu = np.asarray(J_gpu)
    J_ref = np.asarray(J_ref)
    n = J_ref.shape[-1]
    d = (J_ref - J_gpu).reshape(-1, n)
    r = J_ref.reshape(-1, n)
    EL_k = np.linalg.norm(d, axis=0) / np.maximum(np.linalg.norm(r, axis=0), 1e-300)
    Tn = np.linalg.norm(r)
    mask = np.abs(r) >= Tn / C_thresh
    rel = np.where(mask, np.abs(d) / np.where(mask, np.abs(r), 1.0), 0.0)
    EC_k = np.linalg.norm(rel, axis=0)
    return float(np.linalg.norm(EL_k)), float(np.linalg.norm(EC_k))
