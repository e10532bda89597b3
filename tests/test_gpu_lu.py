"""GPU parity of the Newton-matrix LU and solve (the linear algebra Sec. 5
names as the missing piece) against the oracle, through the C ABI.

The Newton matrices of states with tiny species amounts are ill-conditioned
even in the states' own scaling, so on them the checks are the stability
guarantees of LU without pivoting: |L U - P M P^T| <= c N u |L||U| for the
GPU's factors, and a normwise backward error of c N u for the GPU's solves
in the states' scaling.  On well-conditioned matrices in the same pattern the
factors match the oracle's entry by entry and the solves match LAPACK."""
import numpy as np
import pytest

import oracle
import synth
from oracle import linalg as LA
from tests import tiny_mechs as tm
from tests.parity import (equilibrated_backward_ratio, equilibrated_growth, lu_backward_ratio,
                          lu_dense_from_storage, lu_solve_ratio)

pytestmark = pytest.mark.gpu
U64, U32 = 2.0 ** -53, 2.0 ** -24


@pytest.fixture(scope="module")
def pj():
    import paper_1809_01029_gb300 as pj
    from paper_1809_01029_gb300 import build
    build.build()
    pj.load_library()
    return pj


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _mech(mechs, name):
    return getattr(tm, name)() if name in ("all_kinds", "bath_efficiency", "all_types") else mechs(name)


@pytest.mark.parametrize("from_j", [False, True])
@pytest.mark.parametrize("name,n", [("all_kinds", 30), ("all_types", 20), ("h2co13", 100), ("gri53", 40), ("gri53_types", 30), ("usc111", 12)])
def test_lu_fp64_newton_matrices(pj, mechs, name, n, from_j):
    import torch
    m = _mech(mechs, name)
    h = pj.pj_mech_create(m)
    phi, par = synth.make_states(m, n, 800 + n, synth.CONP)
    hs = synth.make_step_sizes(n, 800 + n)
    Jc = oracle.dense_to_csr_values(m, oracle.jacobian(m, synth.CONP, phi, par))
    M = LA.newton_dense(m, Jc, hs, 1.0)
    perm, F, (r, c) = LA.lu_symbolic(m)
    N = M.shape[0]
    if from_j:
        lu = pj.lu_factor(h, dev(Jc), h=dev(hs), gamma=1.0)
    else:
        lu = pj.lu_factor(h, dev(oracle.dense_to_csr_values(m, M)))
    assert lu.dtype == torch.float64 and lu.shape == (len(r), n)
    L, U = lu_dense_from_storage(lu.cpu().numpy(), r, c, N)
    assert lu_backward_ratio(L, U, M[np.ix_(perm, perm)], U64) <= 4.0
    D = np.abs(phi)
    b = np.random.default_rng(n).standard_normal((N, n)) * D
    x = pj.lu_solve(h, lu, dev(b)).cpu().numpy()
    # the solve against the GPU's own factors, whatever their growth
    assert lu_solve_ratio(L, U, x[perm], b[perm], U64) <= 8.0
    # and against M in the states' scaling, within the growth of the factors
    # (about 1 on the workload mechanisms; the tiny all-types mechanism's
    # unphysical thermochemistry gives reverse rates up to 1e45)
    g = np.maximum(equilibrated_growth(L, U, M[np.ix_(perm, perm)], D[perm]), 1.0)
    assert np.all(equilibrated_backward_ratio(M, x, b, D, U64) <= 4.0 * g)
    bb = dev(b)
    pj.lu_solve(h, lu, bb, out=bb)                       # in place
    assert np.array_equal(bb.cpu().numpy(), x)


@pytest.mark.parametrize("name,n", [("gri53", 40), ("usc111", 12)])
def test_lu_fp32_of_the_fp32_newton_matrix(pj, mechs, name, n):
    """The FP32 Newton matrix factored and solved in FP32.  The synthetic
    states are stiff enough that some factorisations leave FP32's range
    (products of factor entries near 1e40); exactly those states are counted
    in the status word, and the others are backward stable at FP32's unit
    roundoff for the FP32 matrix they were given."""
    import torch
    m = mechs(name)
    h = pj.pj_mech_create(m)
    phi, par = synth.make_states(m, n, 900 + n, synth.CONP)
    hs = synth.make_step_sizes(n, 900 + n)
    M32 = pj.newton_matrix_f32(h, synth.CONP, dev(phi), dev(par), dev(hs), 1.0, fmt=pj.PJ_CSR)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    lu = pj.lu_factor(h, M32, status=status)
    assert lu.dtype == torch.float32
    fin = np.all(np.isfinite(lu.cpu().numpy()), axis=0)
    assert int(status.item()) == int((~fin).sum()) < n
    keep = np.flatnonzero(fin)
    lu = lu[:, keep].contiguous()
    phi, M32 = phi[:, keep], M32[:, keep]
    n = len(keep)
    perm, F, (r, c) = LA.lu_symbolic(m)
    N = m.n_species + 1
    row_ptr, col = oracle.csr_pattern(m)
    M = np.zeros((N, N, n))
    M[np.repeat(np.arange(N), np.diff(row_ptr)), col] = M32.cpu().numpy().astype(np.float64)
    L, U = lu_dense_from_storage(lu.cpu().numpy().astype(np.float64), r, c, N)
    assert lu_backward_ratio(L, U, M[np.ix_(perm, perm)], U32, tiny=2.0 ** -149) <= 4.0
    D = np.abs(phi)
    b = (np.random.default_rng(n).standard_normal((N, n)) * D).astype(np.float32)
    x = pj.lu_solve(h, lu, dev(b)).cpu().numpy().astype(np.float64)
    assert np.all(equilibrated_backward_ratio(M, x, b.astype(np.float64), D, U32) <= 4.0)


@pytest.mark.parametrize("name,n", [("all_kinds", 9), ("h2co13", 7), ("gri53", 5), ("usc111", 3), ("ic5874", 2)])
def test_lu_well_conditioned_pattern_matrices(pj, mechs, name, n):
    """Random values in the pattern with a dominant diagonal: factors equal
    the oracle's within the rounding of the same elimination, solves match
    LAPACK.  The 874-species case runs the global-workspace factorisation."""
    m = _mech(mechs, name)
    h = pj.pj_mech_create(m)
    P = oracle.sparsity_pattern(m)
    N = P.shape[0]
    rng = np.random.default_rng(3 + n)
    M = np.where(P[:, :, None], rng.standard_normal((N, N, n)), 0.0)
    M[np.arange(N), np.arange(N)] = np.abs(M).sum(axis=1) + 1.0
    perm, F, st = LA.lu_symbolic(m)
    L, U = LA.lu_factor(M, perm)
    ref = LA.lu_values(L, U, st)
    lu = pj.lu_factor(h, dev(oracle.dense_to_csr_values(m, M))).cpu().numpy()
    r, c = st
    env = np.moveaxis(np.matmul(np.moveaxis(np.abs(L), 2, 0), np.moveaxis(np.abs(U), 2, 0)), 0, 2)[r, c]
    scale = np.where((r < c)[:, None], env, env / np.abs(U[c, c]))
    d = r == c
    scale[d] = env[d] / U[r[d], c[d]] ** 2
    assert np.all(np.abs(lu - ref) <= 4 * N * U64 * scale + 1e-300)
    b = rng.standard_normal((N, n))
    x = pj.lu_solve(h, dev(lu), dev(b)).cpu().numpy()
    xr = LA.solve(M, b)
    assert np.allclose(x, xr, rtol=1e-11, atol=1e-12 * np.abs(xr).max())


def test_lu_zero_pivot_is_counted_and_contained(pj, mechs):
    import torch
    m = mechs("h2co13")
    h = pj.pj_mech_create(m)
    P = oracle.sparsity_pattern(m)
    N = P.shape[0]
    n = 5
    M = np.repeat(np.where(P, 0.1, 0.0)[:, :, None], n, axis=2)
    M[np.arange(N), np.arange(N)] = 3.0
    M[:, :, 2] = 0.0                                       # a zero matrix: first pivot 0
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    lu = pj.lu_factor(h, dev(oracle.dense_to_csr_values(m, M)), status=status).cpu().numpy()
    assert int(status.item()) == 1
    assert np.all(np.isfinite(np.delete(lu, 2, axis=1)))
    e = torch.empty((h.nnz, 0), dtype=torch.float64, device="cuda")
    assert pj.lu_factor(h, e).shape[1] == 0
