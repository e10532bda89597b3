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
