"""Incomplete Cholesky on a given pattern, and its triangular solves.

Test infrastructure (see the package docstring).

Sec. IV.B (eq. (6)) preconditions every contingency matrix with the
factorised base-case matrix B'_basecase.  For a symmetric positive definite
matrix A and a lower-triangular pattern P (containing the diagonal),
incomplete Cholesky computes L with nonzeros only on P such that
    L_ij = (A_ij - sum_{k<j, (i,k) in P, (j,k) in P} L_ik L_jk) / L_jj,  j < i
    L_ii = sqrt(A_ii - sum_{k<i, (i,k) in P} L_ik^2).
With P = the lower triangle of A this is IC(0); with P = the symbolic
Cholesky pattern (all fill) it is the exact Cholesky factor.  Applying the
preconditioner is z = (L L^T)^{-1} r: forward substitution L y = r, then
back substitution L^T z = y.

Pins (tests): (L L^T)_ij = A_ij on P; on a tree-structured matrix IC(0)
equals the dense Cholesky factor; with the full pattern L equals the dense
Cholesky factor; the substitutions invert dense triangular matrices.
"""
from __future__ import annotations

import numpy as np


def ic_on_pattern(A, rows_of_pattern):
    """Incomplete Cholesky of the dense-or-sparse SPD ``A`` on a pattern.

    ``rows_of_pattern[i]`` lists the column indices j <= i of row i of L
    (must contain i).  Returns ``{i: {j: L_ij}}``.
    """
    Ad = A if isinstance(A, dict) else _as_dict(A)
    L = {}
    for i in range(len(rows_of_pattern)):
        cols = sorted(int(c) for c in rows_of_pattern[i])
        assert cols[-1] == i, "pattern row must end at the diagonal"
        Li = {}
        for j in cols:
            s = Ad.get((i, j), 0.0)
            Lj = L[j] if j < i else Li
            for k, lik in Li.items():
                if k < j and k in Lj:
                    s -= lik * Lj[k]
            if j < i:
                Li[j] = s / L[j][j]
            else:
                if s <= 0.0:
                    raise ValueError(f"non-positive pivot at row {i}")
                Li[i] = np.sqrt(s)
        L[i] = Li
    return L


def _as_dict(A):
    A = A.tocoo() if hasattr(A, "tocoo") else None
    if A is None:
        raise TypeError("expected a scipy sparse matrix or a dict")
    return {(int(i), int(j)): float(v) for i, j, v in zip(A.row, A.col, A.data)}


def to_dense(L, n):
    M = np.zeros((n, n))
    for i, row in L.items():
        for j, v in row.items():
            M[i, j] = v
    return M


def forward(L, r):
    """Solve L y = r by forward substitution (row order)."""
    n = r.shape[0]
    y = np.zeros_like(r, dtype=np.float64)
    for i in range(n):
        s = r[i]
        for j, v in L[i].items():
            if j < i:
                s -= v * y[j]
        y[i] = s / L[i][i]
    return y


def backward(L, y):
    """Solve L^T z = y by back substitution (column sweep of L)."""
    n = y.shape[0]
    z = np.array(y, dtype=np.float64)
    for i in range(n - 1, -1, -1):
        z[i] = z[i] / L[i][i]
        for j, v in L[i].items():
            if j < i:
                z[j] -= v * z[i]
    return z


def apply_preconditioner(L, r):
    """z = (L L^T)^{-1} r."""
    return backward(L, forward(L, r))


def symbolic_cholesky(n, lower_pattern):
    """Pattern of the exact Cholesky factor of a matrix whose lower triangle
    has pattern ``lower_pattern`` (fill by graph elimination in index order:
    eliminating vertex k joins all its higher-numbered neighbours)."""
    adj = [set() for _ in range(n)]
    for i in range(n):
        for j in lower_pattern[i]:
            if j != i:
                adj[i].add(int(j))
                adj[int(j)].add(i)
    rows = [set([i]) for i in range(n)]
    for k in range(n):
        hi = sorted(v for v in adj[k] if v > k)
        for a in hi:
            rows[a].add(k)
        for ai in range(len(hi)):
            for bi in range(ai + 1, len(hi)):
                adj[hi[ai]].add(hi[bi])
                adj[hi[bi]].add(hi[ai])
    return [sorted(r) for r in rows]
