"""Reference Kemeny constant of graphs too large for an exact method:
Hutchinson's trace estimator on the pseudo-inverse of the normalised Laplacian.

TEST INFRASTRUCTURE ONLY (see the package docstring).  FP64 throughout.

K = Tr(N^+) with N = I - D^-1/2 A D^-1/2 (Eq. 1).  For a Rademacher vector z,
E[z^T N^+ z] = Tr(N^+), so the mean over independent probes is an unbiased
estimate whose standard error is reported with it (the approximate route the
paper's Sec. 2 mentions for large graphs).  Each probe solves N x = y with
y = z projected off the null vector psi = D^1/2 1 / sqrt(2m) by conjugate
gradients from x = 0, which keeps x in the range of N, so y^T x = z^T N^+ z.
Probes are drawn from numpy's PCG64 with the given seed.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = ["normalized_laplacian", "quad_pinv", "K_hutchinson"]


def normalized_laplacian(g):
    n = g.n
    src = np.repeat(np.arange(n, dtype=np.int64), g.deg)
    dinv = 1.0 / np.sqrt(g.deg.astype(np.float64))
    vals = -dinv[src] * dinv[g.col.astype(np.int64)]
    A = sp.csr_matrix((vals, g.col.astype(np.int64), g.row_off.astype(np.int64)), shape=(n, n))
    return (sp.identity(n, format="csr") + A).tocsr()


def _cg_block(N, Y, tol, maxiter):
    """Plain CG on every column of Y at once (N symmetric positive semidefinite,
    columns of Y in its range).  Returns X with N X = Y column by column."""
    X = np.zeros_like(Y)
    R = Y.copy()
    Pm = R.copy()
    rr = np.einsum("ij,ij->j", R, R)
    stop = (tol ** 2) * np.einsum("ij,ij->j", Y, Y)
    for _ in range(maxiter):
        live = rr > stop
        if not live.any():
            return X
        Q = N @ Pm
        pq = np.einsum("ij,ij->j", Pm, Q)
        alpha = np.where(live, rr / np.where(pq > 0, pq, 1.0), 0.0)
        X += Pm * alpha
        R -= Q * alpha
        rr_new = np.einsum("ij,ij->j", R, R)
        beta = np.where(live, rr_new / np.where(rr > 0, rr, 1.0), 0.0)
        Pm = R + Pm * beta
        rr = rr_new
    raise RuntimeError("CG did not converge")


def quad_pinv(g, Z, tol=1e-10, maxiter=20000, N=None):
    """z^T N^+ z for every column z of Z (n x p)."""
    if N is None:
        N = normalized_laplacian(g)
    psi = np.sqrt(g.deg.astype(np.float64))
    psi /= np.linalg.norm(psi)
    Y = Z - np.outer(psi, psi @ Z)
    X = _cg_block(N, Y, tol, maxiter)
    return np.einsum("ij,ij->j", Y, X)


def K_hutchinson(g, probes: int, seed: int, block: int = 16, tol=1e-10):
    """(mean, standard error, per-probe values) of z^T N^+ z over `probes`
    Rademacher vectors."""
    rng = np.random.default_rng(seed)
    N = normalized_laplacian(g)
    vals = []
    left = probes
    while left > 0:
        b = min(block, left)
        Z = rng.integers(0, 2, size=(g.n, b)).astype(np.float64) * 2.0 - 1.0
        vals.extend(quad_pinv(g, Z, tol=tol, N=N).tolist())
        left -= b
    v = np.asarray(vals)
    se = float(v.std(ddof=1) / np.sqrt(len(v))) if len(v) > 1 else float("inf")
    return float(v.mean()), se, v
