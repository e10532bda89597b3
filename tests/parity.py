"""Comparison helpers for GPU-vs-oracle parity tests.

Floating-point bar: |gpu - ref| <= rtol * max(|ref|, env) + atol, where env is
the oracle's absolute envelope (the sum of magnitudes of the terms that make
up the value; near chemical equilibrium net rates are differences of nearly
equal forward and reverse rates, Sec. 3.2, so a correct evaluation can only
be held to the rounding of those terms).  rtol = 1e-10, atol = 1e-20 for
source terms; rtol = 1e-8 per Jacobian entry.  Entries whose envelope is at
most 10 |ref| (no significant cancellation) must in addition meet the plain
per-entry bar |gpu - ref| <= rtol |ref| + atol.  Every check records how many
entries passed only through the envelope; the test session prints the
totals (tests/conftest.py).
"""
import contextlib
import os

import numpy as np

RTOL_SRC, ATOL_SRC = 1e-10, 1e-20
RTOL_JAC, ATOL_JAC = 1e-8, 1e-20

# Stated accuracy of the FP32 Newton matrix M = I - h gamma J against the
# FP64 oracle, per entry: |dM| <= NEWTON_ENTRY (|M| + h gamma env(J)) +
# NEWTON_FLOOR.  The floor is FP32's normal range: below 2^-126 a binary32
# value keeps fewer significant bits, and the FP32 L2 reductions that sum the
# entries flush subnormal contributions to zero; next to M's unit diagonal
# such entries carry no weight in a Newton step.
NEWTON_ENTRY = 1e-5
NEWTON_FLOOR = 64 * 2.0 ** -126


def newton_tol(scale):
    return NEWTON_ENTRY * np.asarray(scale) + NEWTON_FLOOR


# the FP32 Newton form's measured error against the FP64 oracle, one record
# per check (printed at the end of the test session)
NEWTON_REPORT = []


def newton_error(got, ref, scale, what=""):
    """Record the error of FP32 Newton-matrix values `got` against the
    oracle's M = I - h gamma J (`ref`, entries x states) in the terms of the
    stated accuracy: per entry |dM| / (|M| + h gamma env(J)) (`scale`), and
    per state the Frobenius error ||dM||_F / ||M||_F."""
    got, ref, scale = (np.asarray(a, dtype=np.float64) for a in (got, ref, scale))
    err = np.abs(got - ref)
    rel = err / np.maximum(scale, NEWTON_FLOOR)
    frob = np.sqrt((err ** 2).sum(axis=0)) / np.sqrt((ref ** 2).sum(axis=0))
    rec = dict(what=what, entries=int(err.size), states=int(err.shape[-1]),
               entry_median=float(np.median(rel)), entry_p99=float(np.quantile(rel, 0.99)),
               entry_max=float(rel.max()), frob_median=float(np.median(frob)), frob_max=float(frob.max()))
    NEWTON_REPORT.append(rec)
    return rec


# one record per check_close call: what, entries, entries that passed only
# through the envelope, well-conditioned entries, largest relative error of a
# well-conditioned entry
REPORT = []
WELL = 10.0     # env <= WELL |ref|: an entry without significant cancellation


def check_close(got, ref, env, rtol, atol, what="", max_env_frac=None):
    """got within rtol * max(|ref|, env) + atol of ref, entry by entry; the
    well-conditioned entries (env <= WELL |ref|) also within rtol |ref| +
    atol.  Returns how many entries passed only through the envelope; with
    max_env_frac, at most that fraction of the entries (and at least one)
    may."""
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
    plain = rtol * np.abs(ref) + atol
    well = env <= WELL * np.abs(ref)
    strict_bad = well & ~(err <= plain)
    if strict_bad.any():
        idx = np.unravel_index(np.argmax(np.where(strict_bad, err / np.maximum(plain, 1e-300), 0)), err.shape)
        raise AssertionError(
            f"{what}: {strict_bad.sum()} well-conditioned entries (env <= {WELL} |ref|) beyond rtol |ref| + atol; "
            f"worst at {idx}: gpu={got[idx]!r} ref={ref[idx]!r} env={env[idx]!r} err={err[idx]!r}")
    needed_env = int(np.sum(err > plain))
    rel_well = np.where(well & (ref != 0), err / np.where(ref != 0, np.abs(ref), 1.0), 0.0)
    REPORT.append(dict(what=what, entries=int(err.size), needed_env=needed_env, well=int(well.sum()),
                       worst_rel_well=float(rel_well.max()) if rel_well.size else 0.0))
    if max_env_frac is not None:
        assert needed_env <= max(1, max_env_frac * err.size), f"{what}: {needed_env} of {err.size} entries " \
                                                              "passed only through the envelope"
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


def lu_dense_from_storage(vals, rows, cols, N):
    """(L unit lower, U upper) [N, N, n] from factor values in storage order
    (1 / U_kk in the diagonal slots)."""
    n = vals.shape[1]
    L = np.zeros((N, N, n))
    U = np.zeros((N, N, n))
    low = rows > cols
    L[rows[low], cols[low]] = vals[low]
    L[np.arange(N), np.arange(N)] = 1.0
    up = rows < cols
    U[rows[up], cols[up]] = vals[up]
    d = rows == cols
    U[rows[d], cols[d]] = 1.0 / vals[d]
    return L, U


def lu_backward_ratio(L, U, A, u, tiny=2.0 ** -1074):
    """max over entries of |L U - A| / (N u (|L||U|) + tiny (row sums of |L|
    + column sums of |U| + 1)): at most a small constant for a backward-stable
    factorisation (computed in float64).  The tiny term (the subnormal
    spacing of the factors' precision) covers gradual underflow of factor
    entries, which the relative bound alone does not."""
    N = A.shape[0]
    mm = lambda a, b: np.moveaxis(np.matmul(np.moveaxis(a, 2, 0), np.moveaxis(b, 2, 0)), 0, 2)
    LU = mm(L, U)
    env = mm(np.abs(L), np.abs(U))
    under = tiny * (np.abs(L).sum(axis=1)[:, None, :] + np.abs(U).sum(axis=0)[None, :, :] + 1.0)
    r = np.abs(LU - A)
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.where(r == 0, 0.0, r / (N * u * env + under))
    return float(q.max())


def equilibrated_backward_ratio(M, x, b, D, u):
    """Normwise backward error of M x = b in the variables scaled by D (the
    states' own magnitudes, rows and columns), over N u, per state."""
    N = M.shape[0]
    At = M * D[None, :, :] / D[:, None, :]
    xt, bt = x / D, b / D
    r = np.abs(np.einsum("ijn,jn->in", At, xt) - bt).max(axis=0)
    den = np.abs(At).sum(axis=1).max(axis=0) * np.abs(xt).max(axis=0) + np.abs(bt).max(axis=0)
    return r / den / (N * u)


def lu_solve_ratio(L, U, xp, bp, u):
    """Residual of the computed solution against the computed factors, in
    pivot order (xp = x[perm], bp = b[perm]): max |L U x - b| / (N u (|L||U||x|
    + |b|)).  Triangular substitution is componentwise backward stable, so
    this is a small constant whatever the growth of the factors."""
    N = L.shape[0]
    mv = lambda A, v: np.einsum("ijn,jn->in", A, v)
    r = np.abs(mv(L, mv(U, xp)) - bp)
    env = mv(np.abs(L), mv(np.abs(U), np.abs(xp))) + np.abs(bp)
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.where(r == 0, 0.0, r / (N * u * env))
    return float(q.max())


def equilibrated_growth(L, U, A, Dp):
    """Per state, the growth of LU in the scaled variables (Dp: the states'
    magnitudes in pivot order): || |L||U| ||_inf / ||A||_inf after scaling rows
    by 1/Dp and columns by Dp."""
    mm = lambda a, b: np.moveaxis(np.matmul(np.moveaxis(a, 2, 0), np.moveaxis(b, 2, 0)), 0, 2)
    sc = Dp[None, :, :] / Dp[:, None, :]
    E = mm(np.abs(L), np.abs(U)) * sc
    return E.sum(axis=1).max(axis=0) / (np.abs(A) * sc).sum(axis=1).max(axis=0)


def y_envelope(m, mode, phi, par):
    """Absolute rounding envelope of y = (wdot, dT/dt): per species the sum of
    |nu| (|q'| + |q''|) over the reactions that change it, and the source-term
    envelope of dT/dt."""
    import oracle
    r = oracle.rates(m, mode, phi, par)
    _, fenv = oracle.source_term_envelope(m, mode, phi, par)
    nu = r["nu"]
    ew = np.zeros_like(r["wdot"])
    for i in range(m.n_reactions):
        t = np.abs(r["qf"][i]) + np.abs(r["qr"][i])
        for k in range(m.n_species):
            if nu[k, i]:
                ew[k] += abs(nu[k, i]) * t
    return np.concatenate([ew, fenv[:1]], axis=0)


@contextlib.contextmanager
def jacobian_layout(name):
    """Run the library's Jacobian entries with one kernel family: "coop" (the
    warps of a block share 32 states; L2-resident accumulation, rounding
    depends on the order of cross-warp reductions), "coop-global" (the same
    with the tile's per-state arrays in the workspace instead of shared
    memory) or "percore" (one state per thread; bit-reproducible).  The
    library reads PYJAC_GB_JAC_LAYOUT and PYJAC_GB_COOP_ARRAYS at every
    launch."""
    keys = ("PYJAC_GB_JAC_LAYOUT", "PYJAC_GB_COOP_ARRAYS")
    old = {k: os.environ.get(k) for k in keys}
    os.environ["PYJAC_GB_JAC_LAYOUT"] = "coop" if name.startswith("coop") else name
    if name == "coop-global":
        os.environ["PYJAC_GB_COOP_ARRAYS"] = "global"
    else:
        os.environ.pop("PYJAC_GB_COOP_ARRAYS", None)
    try:
        yield
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v