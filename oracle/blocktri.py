"""Exact Kemeny constant of graphs whose Laplacian is block tridiagonal: a
w x h grid (any subset of its edges) numbered row by row, vertex y * w + x.

TEST INFRASTRUCTURE ONLY (see the package docstring).  FP64 throughout.

Eq. (1) defines K as the sum of the reciprocals of the non-zero eigenvalues
of I - D^-1/2 A D^-1/2, i.e. the trace of its pseudo-inverse.  Grounding the
Laplacian at r (deleting row and column r) gives the same number as

    K = sum_{i != r} d_i (L_r^-1)_ii  -  d_r^T L_r^-1 d_r / (2m)

(L^+ = Pi L_r^-1 Pi with Pi the projector off the constant vector; this is
Eq. (3) with the minus sign, evaluated at v = r).  For a row-major grid, L_r
with r the last vertex is block tridiagonal with h blocks of w rows (the last
one w - 1), and both terms need only the diagonal blocks of L_r^-1 and one
solve.  They come from the textbook block recurrences of selected inversion
(no fill outside the band):

    S_0 = A_00,   S_i = A_ii - C_{i-1}^T S_{i-1}^-1 C_{i-1}          (forward)
    G_last = S_last^-1,
    G_i = S_i^-1 + S_i^-1 C_i G_{i+1} C_i^T S_i^-1                   (backward)

with C_i = A_{i,i+1} and G_i the i-th diagonal block of A^-1, and the block
Thomas solve for A x = d.  The cost is O(h w^3) flops and O(h w^2) memory
(1000 x 1000 grid: about 10^13 flops, 8 GB).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = ["K_block_tridiagonal"]


def _blocks(g, w: int):
    """Diagonal and upper off-diagonal blocks of the Laplacian grounded at the
    last vertex, as dense arrays; raises if some edge spans more than one block."""
    n = g.n
    if n % w != 0 or n < 2 * w:
        raise ValueError("n must be a multiple of the block width, with at least two blocks")
    src = np.repeat(np.arange(n, dtype=np.int64), g.deg)
    dst = g.col.astype(np.int64)
    if np.any(np.abs(src // w - dst // w) > 1):
        raise ValueError("Laplacian is not block tridiagonal for this block width")
    L = sp.csr_matrix((-np.ones(src.shape[0]), (src, dst)), shape=(n, n))
    L = (L + sp.diags(g.deg.astype(np.float64))).tocsr()
    m = n - 1  # grounded size: the last vertex is removed
    h = n // w
    sizes = [w] * (h - 1) + [w - 1]
    starts = [i * w for i in range(h)]
    A = [L[s:s + z, s:s + z].toarray() for s, z in zip(starts, sizes)]
    C = [L[starts[i]:starts[i] + sizes[i], starts[i + 1]:starts[i + 1] + sizes[i + 1]].toarray()
         for i in range(h - 1)]
    d = g.deg.astype(np.float64)[:m]
    return A, C, [d[s:s + z] for s, z in zip(starts, sizes)]


def _inv_spd(M):
    X = np.linalg.inv(M)
    return 0.5 * (X + X.T)


def K_block_tridiagonal(g, w: int) -> float:
    """Exact K (Eq. 1) of a graph on vertices 0..n-1 whose edges join only
    vertices of the same or adjacent blocks of w consecutive ids, grounded at
    r = n - 1.  Returns a Python float."""
    A, C, d = _blocks(g, w)
    h = len(A)
    # forward sweep: inverses of the Schur complements
    Sinv = [None] * h
    S = A[0]
    for i in range(h):
        if i > 0:
            T = Sinv[i - 1] @ C[i - 1]
            S = A[i] - C[i - 1].T @ T
        Sinv[i] = _inv_spd(S)
    # block Thomas solve of L_r x = d_r
    z = [None] * h
    z[0] = d[0].copy()
    for i in range(1, h):
        z[i] = d[i] - C[i - 1].T @ (Sinv[i - 1] @ z[i - 1])
    x = [None] * h
    x[h - 1] = Sinv[h - 1] @ z[h - 1]
    for i in range(h - 2, -1, -1):
        x[i] = Sinv[i] @ (z[i] - C[i] @ x[i + 1])
    quad = float(sum(np.dot(d[i], x[i]) for i in range(h)))
    # backward sweep: diagonal blocks of L_r^-1, only their diagonals are kept
    G = Sinv[h - 1]
    tr = float(np.dot(d[h - 1], np.diag(G)))
    for i in range(h - 2, -1, -1):
        T = Sinv[i] @ C[i]
        G = Sinv[i] + T @ G @ T.T
        tr += float(np.dot(d[i], np.diag(G)))
        Sinv[i + 1] = None  # free as we go
    return tr - quad / (2.0 * g.m)
