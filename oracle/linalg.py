"""CPU oracle for the implicit-step linear algebra that consumes the Jacobian:
LU factorisation and solve of the Newton matrix M = I - h gamma J in the
Jacobian's fixed pattern (the step the paper names as the missing piece for
an implicit integrator, Sec. 5; Sec. 3.4 motivates the approximate form by
such solvers reusing one factorisation).

TEST INFRASTRUCTURE ONLY (same rules as ``oracle.kinetics``).

The method is fixed here, since the paper gives none:
* ordering: the species block is ordered by greedy minimum degree on the
  symmetrised pattern (A + A^T without the diagonal) -- repeatedly take the
  remaining species with the fewest remaining neighbours in the elimination
  graph (ties: the lowest species index), then join its remaining neighbours
  into a clique; T and S (dense rows and columns) come last.  perm[k] is the
  state-vector index of the k-th pivot;
* factorisation without pivoting of A = P M P^T (A[k, l] = M[perm[k],
  perm[l]]): A = L U, L unit lower triangular, U upper triangular (Doolittle);
* symbolic pattern F: the structure of A plus the fill of eliminating it in
  that order; storage order: the strictly lower rows k = 0 .. N-1 (columns
  ascending), then the upper rows k = N-1 .. 0, each as 1 / U[k, k] followed
  by U[k, j > k] (columns ascending) -- the order in which forward and
  backward substitution read them;
* solve: x with M x = b.
"""
from __future__ import annotations

import numpy as np

from .kinetics import EXACT, sparsity_pattern


def min_degree_order(S):
    """Greedy minimum-degree elimination order of the graph with symmetric
    adjacency S [m, m] (the diagonal ignored): repeatedly the remaining
    vertex with the fewest remaining neighbours (ties: lowest index), whose
    remaining neighbours then become a clique."""
    m = S.shape[0]
    adj = [set(np.flatnonzero(S[i])) - {i} for i in range(m)]
    alive = set(range(m))
    order = []
    while alive:
        k = min(alive, key=lambda v: (len(adj[v] & alive), v))
        nb = adj[k] & alive
        for a in nb:
            adj[a] |= nb - {a}
        alive.remove(k)
        order.append(k)
    return order


def lu_ordering(mech, form=EXACT):
    """perm [N]: greedy minimum-degree species order, then T (0) and S (1)."""
    P = sparsity_pattern(mech, form)
    S = P[2:, 2:] | P[2:, 2:].T
    return np.array([2 + k for k in min_degree_order(S)] + [0, 1], dtype=np.int32)


def symbolic_fill(A):
    """Structure [N, N] of L + U for LU without pivoting of a matrix with
    structure A (in pivot order): A plus the fill of each elimination."""
    F = A.copy()
    N = F.shape[0]
    for k in range(N):
        rows = np.flatnonzero(F[k + 1:, k]) + k + 1
        cols = np.flatnonzero(F[k, k + 1:]) + k + 1
        F[np.ix_(rows, cols)] = True
    return F


def lu_symbolic(mech, form=EXACT):
    """(perm, F [N, N] bool in pivot order, storage (rows, cols) in pivot
    order) of the factorisation described in the module notes."""
    perm = lu_ordering(mech, form)
    P = sparsity_pattern(mech, form)
    F = symbolic_fill(P[np.ix_(perm, perm)])
    N = F.shape[0]
    r, c = [], []
    for k in range(N):
        for j in range(k):
            if F[k, j]:
                r.append(k)
                c.append(j)
    for k in range(N - 1, -1, -1):
        r.append(k)
        c.append(k)
        for j in range(k + 1, N):
            if F[k, j]:
                r.append(k)
                c.append(j)
    return perm, F, (np.array(r, dtype=np.int32), np.array(c, dtype=np.int32))


def newton_dense(mech, J_csr_vals, h, gamma, form=EXACT):
    """Dense M = I - h gamma J [N, N, n] from CSR values of J."""
    from .kinetics import csr_pattern
    row_ptr, col = csr_pattern(mech, form)
    N = len(row_ptr) - 1
    n = J_csr_vals.shape[1]
    J = np.zeros((N, N, n))
    rows = np.repeat(np.arange(N), np.diff(row_ptr))
    J[rows, col] = J_csr_vals
    M = -(np.asarray(h) * gamma) * J
    M[np.arange(N), np.arange(N)] += 1.0
    return M


def lu_factor(M, perm):
    """LU without pivoting of A = P M P^T for every state by Gaussian
    elimination: at pivot k, l_ik = a_ik / a_kk and a_ij -= l_ik a_kj for
    i, j > k.  Returns (L [N, N, n] unit lower, U [N, N, n] upper)."""
    A = M[np.ix_(perm, perm)].astype(np.float64).copy()
    N = A.shape[0]
    for k in range(N):
        A[k + 1:, k] = A[k + 1:, k] / A[k, k]
        A[k + 1:, k + 1:] -= A[k + 1:, k][:, None] * A[k, k + 1:][None, :]
    eye = np.eye(N)[:, :, None]
    low = np.tril(np.ones((N, N)), -1)[:, :, None]
    return low * A + eye, np.triu(np.ones((N, N)))[:, :, None] * A


def lu_values(L, U, storage):
    """Factor values [lu_nnz, n] in storage order (1 / U[k, k] on the
    diagonal slots)."""
    r, c = storage
    out = np.where((r < c)[:, None], U[r, c], L[r, c])
    diag = r == c
    out[diag] = 1.0 / U[r[diag], c[diag]]
    return out


def solve(M, b):
    """x with M x = b per state (LAPACK through numpy)."""
    return np.linalg.solve(np.moveaxis(M, 2, 0), np.moveaxis(b, 1, 0)[..., None])[..., 0].T
