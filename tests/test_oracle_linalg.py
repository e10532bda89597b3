"""Pins of the oracle's Newton-matrix linear algebra (oracle/linalg.py):
orderings whose fill is known, the symbolic fill as the closure of the
elimination, a factorisation worked by hand, L U = P M P^T, and solves
against LAPACK."""
import numpy as np
import pytest

import oracle
import synth
from oracle import linalg as LA
from tests.parity import equilibrated_backward_ratio, lu_backward_ratio, lu_dense_from_storage

U64 = 2.0 ** -53


def _fill(S, order):
    A = S[np.ix_(order, order)].copy()
    np.fill_diagonal(A, True)
    return int(LA.symbolic_fill(A).sum() - A.sum())


def test_min_degree_on_arrow_and_path_gives_no_fill():
    """An arrowhead (one hub joined to every leaf) eliminated leaves first,
    and a path eliminated from its ends, factor without fill."""
    m = 9
    arrow = np.zeros((m, m), dtype=bool)
    arrow[0, :] = arrow[:, 0] = True
    o = LA.min_degree_order(arrow)
    # leaves 1..7 first; hub and last leaf tie at degree 1 (lowest index wins)
    assert o == list(range(1, m - 1)) + [0, m - 1] and _fill(arrow, o) == 0
    assert _fill(arrow, list(range(m))) == (m - 1) * (m - 2)    # hub first fills everything
    path = np.zeros((m, m), dtype=bool)
    for i in range(m - 1):
        path[i, i + 1] = path[i + 1, i] = True
    o = LA.min_degree_order(path)
    assert o[0] == 0 and _fill(path, o) == 0


def test_min_degree_picks_lowest_degree_then_lowest_index():
    S = np.zeros((5, 5), dtype=bool)
    for a, b in ((0, 1), (0, 2), (0, 3), (1, 2), (3, 4)):
        S[a, b] = S[b, a] = True
    # degrees 3, 2, 2, 2, 1: vertex 4 first; then 3 (degree 1 after 4 goes)
    assert LA.min_degree_order(S)[:2] == [4, 3]


@pytest.mark.parametrize("name", ["h2co13", "gri53"])
def test_symbolic_fill_is_the_closure_of_elimination(name):
    m = synth.make_mechanism(name)
    perm, F, (r, c) = LA.lu_symbolic(m)
    N = F.shape[0]
    assert sorted(perm) == list(range(N)) and list(perm[-2:]) == [0, 1]
    P = oracle.sparsity_pattern(m)
    assert np.all(F[P[np.ix_(perm, perm)]])
    # closure: F[i,k] and F[k,j] with k < i, j imply F[i,j]
    for k in range(N):
        rows = np.flatnonzero(F[k + 1:, k]) + k + 1
        cols = np.flatnonzero(F[k, k + 1:]) + k + 1
        assert np.all(F[np.ix_(rows, cols)])
    # every fill entry has a generating pivot
    fill = F & ~P[np.ix_(perm, perm)]
    for i, j in zip(*np.nonzero(fill)):
        k = np.arange(min(i, j))
        assert np.any(F[i, k] & F[k, j])
    # storage: each F entry once; lower rows ascending, then upper rows descending
    assert len(r) == F.sum() and np.all(F[r, c])
    nl = int((r > c).sum())
    assert np.all(r[:nl] > c[:nl]) and np.all(np.diff(r[:nl]) >= 0)
    assert np.all(np.diff(r[nl:]) <= 0) and np.all(r[nl:] <= c[nl:])


def test_factorisation_by_hand():
    M = np.array([[4.0, 1.0, 0.0], [2.0, 3.0, 1.0], [0.0, 1.0, 2.0]])[:, :, None]
    L, U = LA.lu_factor(M, np.arange(3))
    assert np.allclose(L[:, :, 0], [[1, 0, 0], [0.5, 1, 0], [0, 0.4, 1]], rtol=1e-15)
    assert np.allclose(U[:, :, 0], [[4, 1, 0], [0, 2.5, 1], [0, 0, 1.6]], rtol=1e-15)


@pytest.mark.parametrize("name", ["h2co13", "gri53"])
def test_newton_matrix_factors_and_solves(name):
    m = synth.make_mechanism(name)
    n = 6
    phi, par = synth.make_states(m, n, 71, synth.CONP)
    hs = synth.make_step_sizes(n, 71)
    J = oracle.jacobian(m, synth.CONP, phi, par)
    M = oracle.newton_matrix(m, synth.CONP, phi, par, hs)
    Mn = LA.newton_dense(m, oracle.dense_to_csr_values(m, J), hs, 1.0)
    assert np.array_equal(Mn, M)
    perm, F, st = LA.lu_symbolic(m)
    L, U = LA.lu_factor(M, perm)
    N = M.shape[0]
    A = M[np.ix_(perm, perm)]
    LU = np.einsum("ikn,kjn->ijn", L, U)
    env = np.einsum("ikn,kjn->ijn", np.abs(L), np.abs(U))
    assert np.all(np.abs(LU - A) <= 4 * N * U64 * env)
    assert np.all(L[~F] == 0) and np.all(U[~F] == 0)
    assert np.all(np.triu(np.ones((N, N)), 1)[:, :, None] * L == 0)
    vals = LA.lu_values(L, U, st)
    assert vals.shape == (F.sum(), n)
    # substitution with the stored factors; the Newton matrices of states
    # with tiny species amounts are ill-conditioned even after scaling by the
    # state's magnitudes (kappa ~ 1e20), so the check is the normwise backward
    # error in those scaled variables, which LAPACK's solution meets too
    b = np.random.default_rng(5).standard_normal((N, n)) * np.abs(phi)
    x = np.empty_like(b)
    r, c = st
    for s in range(n):
        y = np.zeros(N)
        for k in range(N):
            y[k] = b[perm[k], s] - sum(vals[e, s] * y[c[e]] for e in np.flatnonzero((r == k) & (c < k)))
        z = np.zeros(N)
        for k in range(N - 1, -1, -1):
            up = np.flatnonzero((r == k) & (c > k))
            d = np.flatnonzero((r == k) & (c == k))[0]
            z[k] = (y[k] - sum(vals[e, s] * z[c[e]] for e in up)) * vals[d, s]
        x[perm, s] = z
    D = np.abs(phi)
    assert np.all(equilibrated_backward_ratio(M, x, b, D, U64) <= 4.0)
    assert np.all(equilibrated_backward_ratio(M, LA.solve(M, b), b, D, U64) <= 4.0)
    # a wrong substitution (the diagonal slot used as U_kk, not its inverse) fails it
    x_bad = x.copy()
    x_bad[perm[0]] *= 1.5
    assert not np.all(equilibrated_backward_ratio(M, x_bad, b, D, U64) <= 4.0)


def test_diagonally_dominant_pattern_matrix_factors_match_by_hand_elimination():
    """On a well-conditioned matrix in the pattern, the factors from the
    storage order reproduce A and the solve matches LAPACK closely."""
    m = synth.make_mechanism("h2co13")
    perm, F, st = LA.lu_symbolic(m)
    P = oracle.sparsity_pattern(m)
    N = P.shape[0]
    rng = np.random.default_rng(9)
    M = np.where(P[:, :, None], rng.standard_normal((N, N, 3)), 0.0)
    M[np.arange(N), np.arange(N)] = np.abs(M).sum(axis=1) + 1.0
    L, U = LA.lu_factor(M, perm)
    vals = LA.lu_values(L, U, st)
    L2, U2 = lu_dense_from_storage(vals, st[0], st[1], N)
    assert lu_backward_ratio(L2, U2, M[np.ix_(perm, perm)], U64) <= 4.0
    b = rng.standard_normal((N, 3))
    x = LA.solve(M, b)
    assert np.allclose(np.einsum("ijn,jn->in", M, x), b, rtol=0, atol=1e-13 * np.abs(b).max())
