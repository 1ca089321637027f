"""Exact Kemeny constants, closed forms, spanning-tree enumeration and the
literal path-mapping definition.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Everything here is
FP64 or exact rational/integer arithmetic.
"""
from __future__ import annotations

import itertools
import math
from collections import deque

import numpy as np

__all__ = [
    "laplacian_dense", "K_dense", "K_grounded", "K_eq3", "K_closed", "K_tree_graph",
    "trace_green", "resistance", "resistance_sparse", "resistance_all_edges", "spanning_trees", "kirchhoff_count",
    "orient", "f_literal", "two_forests", "K_forest_formula", "hoeffding_trees",
    "K_torus", "K_hypercube",
]


def laplacian_dense(g) -> np.ndarray:
    n = g.n
    L = np.zeros((n, n), dtype=np.float64)
    src = np.repeat(np.arange(n), g.deg)
    L[src, g.col] = -1.0
    L[np.arange(n), np.arange(n)] = g.deg.astype(np.float64)
    return L


def K_dense(g) -> float:
    """Eq. (1): K = Tr(Lnorm^+) = sum_{i>=2} 1/sigma_i, Lnorm = I - D^-1/2 A D^-1/2."""
    L = laplacian_dense(g)
    dinv = 1.0 / np.sqrt(g.deg.astype(np.float64))
    N = L * dinv[:, None] * dinv[None, :]
    w = np.linalg.eigvalsh(N)
    w.sort()
    return float(np.sum(1.0 / w[1:]))


def K_grounded(g, r: int = 0) -> float:
    """K = sum_{i != r} d_i (L_r^-1)_ii - d_r^T L_r^-1 d_r / (2m), L_r the Laplacian with
    row and column r removed, d_r the degree vector without entry r.  Follows from
    L^+ = Pi L_r^-1 Pi and equals Eq. (3) with the minus sign
    (Tr(I - P_r)^-1 - (Lnorm^+)_rr / pi_r)."""
    L = laplacian_dense(g)
    keep = np.arange(g.n) != r
    Lr = L[np.ix_(keep, keep)]
    d = g.deg.astype(np.float64)[keep]
    X = np.linalg.inv(Lr)
    return float(np.dot(d, np.diag(X)) - d @ X @ d / (2.0 * g.m))


def trace_green(g, r: int) -> float:
    """Tr(I - P_r)^-1 = sum_{i != r} d_i (L_r^-1)_ii: the expected number of steps of
    Wilson's algorithm rooted at r (Sec. 2.2 and the proof of Theorem 8)."""
    L = laplacian_dense(g)
    keep = np.arange(g.n) != r
    X = np.linalg.inv(L[np.ix_(keep, keep)])
    return float(np.dot(g.deg.astype(np.float64)[keep], np.diag(X)))


def K_eq3(g, v: int, sign: float) -> float:
    """Eq. (3) as printed (sign=+1) or corrected (sign=-1):
    Tr(I - P_v)^-1 +/- (Lnorm^+)_vv / pi_v."""
    L = laplacian_dense(g)
    dinv = 1.0 / np.sqrt(g.deg.astype(np.float64))
    N = L * dinv[:, None] * dinv[None, :]
    Np = np.linalg.pinv(N, hermitian=True)
    pi_v = g.deg[v] / (2.0 * g.m)
    return trace_green(g, v) + sign * Np[v, v] / pi_v


def K_closed(family: str, *args) -> float:
    """Closed forms of K for standard families (normalised-Laplacian spectra)."""
    if family == "complete":
        (n,) = args
        return (n - 1) ** 2 / n
    if family == "cycle":
        (n,) = args
        return (n * n - 1) / 6.0
    if family == "star":
        (n,) = args
        return n - 1.5
    if family == "complete_bipartite":
        a, b = args
        return a + b - 1.5
    raise KeyError(family)


def K_torus(a: int, b: int) -> float:
    """a x b torus (4-regular): eigenvalues 1 - (cos 2pi j/a + cos 2pi k/b)/2."""
    j = np.arange(a)[:, None]
    k = np.arange(b)[None, :]
    lam = 1.0 - (np.cos(2 * np.pi * j / a) + np.cos(2 * np.pi * k / b)) / 2.0
    lam = lam.ravel()[1:]
    return float(np.sum(1.0 / lam))


def K_hypercube(k: int) -> float:
    """Q_k: eigenvalues 2j/k with multiplicity C(k, j)."""
    return float(sum(math.comb(k, j) * k / (2.0 * j) for j in range(1, k + 1)))


def K_tree_graph(g) -> float:
    """G itself a tree: the only spanning tree is G, so the 2-forest sum of
    Theorem 1's proof is over single-edge removals:
    K = (1/2m) sum_e vol_e (2m - vol_e)."""
    assert g.m == g.n - 1
    n = g.n
    parent = -np.ones(n, dtype=np.int64)
    order = [0]
    seen = np.zeros(n, dtype=bool)
    seen[0] = True
    dq = deque([0])
    while dq:
        u = dq.popleft()
        for w in g.neighbors(u):
            if not seen[w]:
                seen[w] = True
                parent[w] = u
                order.append(int(w))
                dq.append(int(w))
    vol = g.deg.astype(np.int64).copy()
    for v in reversed(order[1:]):
        vol[parent[v]] += vol[v]
    twom = 2 * g.m
    return float(sum(int(vol[v]) * (twom - int(vol[v])) for v in order[1:])) / twom


def resistance(g, u: int, v: int) -> float:
    """Effective resistance (e_u - e_v)^T L^+ (e_u - e_v), grounded at u."""
    L = laplacian_dense(g)
    keep = np.arange(g.n) != u
    X = np.linalg.inv(L[np.ix_(keep, keep)])
    idx = int(v) - (1 if v > u else 0)
    return float(X[idx, idx])


def resistance_sparse(g, u: int, v: int, rtol: float = 1e-13) -> float:
    """Effective resistance (e_u - e_v)^T L^+ (e_u - e_v) for graphs too large
    for a dense inverse: the Laplacian grounded at u (SPD) solved for e_v by
    scipy's conjugate gradients with the diagonal preconditioner, R = x_v."""
    import scipy.sparse as sp
    from scipy.sparse.linalg import LinearOperator, cg

    n = g.n
    rows = np.repeat(np.arange(n), np.diff(g.row_off))
    A = sp.csr_matrix((np.ones(len(g.col)), (rows, g.col)), shape=(n, n))
    L = sp.diags(np.asarray(A.sum(axis=1)).ravel()) - A
    keep = np.arange(n) != u
    Lg = L[keep][:, keep].tocsr()
    b = np.zeros(n - 1)
    b[int(v) - (1 if v > u else 0)] = 1.0
    dinv = 1.0 / Lg.diagonal()
    M = LinearOperator(Lg.shape, matvec=lambda x: dinv * x)
    x, info = cg(Lg, b, rtol=rtol, atol=0.0, maxiter=50 * n + 1000, M=M)
    if info != 0:
        raise RuntimeError("CG did not converge")
    return float(x[int(v) - (1 if v > u else 0)])


def resistance_all_edges(g) -> dict:
    L = laplacian_dense(g)
    Lp = np.linalg.pinv(L, hermitian=True)
    out = {}
    for a, b in g.edges():
        out[(int(a), int(b))] = float(Lp[a, a] + Lp[b, b] - 2 * Lp[a, b])
    return out


def kirchhoff_count(g) -> float:
    """Matrix-tree theorem: number of spanning trees = det(L_0)."""
    L = laplacian_dense(g)
    return float(np.linalg.det(L[1:, 1:]))


def spanning_trees(g):
    """All spanning trees of a tiny graph, as lists of undirected edges (u < v)."""
    E = [tuple(map(int, e)) for e in g.edges()]
    n = g.n
    out = []
    for comb in itertools.combinations(range(len(E)), n - 1):
        par = list(range(n))

        def find(x):
            while par[x] != x:
                par[x] = par[par[x]]
                x = par[x]
            return x

        ok = True
        for i in comb:
            a, b = E[i]
            ra, rb = find(a), find(b)
            if ra == rb:
                ok = False
                break
            par[ra] = rb
        if ok:
            out.append([E[i] for i in comb])
    return out


def orient(n: int, edges, r: int) -> np.ndarray:
    """Parent array of the tree `edges` rooted at r (parent[r] = -1)."""
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    parent = -np.ones(n, dtype=np.int32)
    seen = [False] * n
    seen[r] = True
    dq = deque([r])
    while dq:
        u = dq.popleft()
        for w in adj[u]:
            if not seen[w]:
                seen[w] = True
                parent[w] = u
                dq.append(w)
    return parent


def _component(n, edges, start):
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    seen = {start}
    dq = deque([start])
    while dq:
        u = dq.popleft()
        for w in adj[u]:
            if w not in seen:
                seen.add(w)
                dq.append(w)
    return seen


def f_literal(g, r: int, p0: np.ndarray, parent: np.ndarray, u_only=None) -> int:
    """f(tau) straight from Definition 1 and Theorem 3: for each u != r, take the
    tau0 path P_u = (u -> p0(u) -> ... -> r) and the tau path from u to r; for every
    directed P_u edge that the tau path uses in the same direction build the
    2-forest tau \\ e and add vol(T1) (component of r); for every P_u edge that the
    tau path uses reversed subtract vol(T1); weight by d(u).  With `u_only` the
    sum is restricted to that single u."""
    n = g.n
    deg = g.deg
    tedges = [(int(v), int(parent[v])) for v in range(n) if v != r]
    f = 0
    for u in (range(n) if u_only is None else [int(u_only)]):
        if u == r:
            continue
        P = set()
        x = u
        while x != r:
            P.add((x, int(p0[x])))
            x = int(p0[x])
        Pt = []
        y = u
        while y != r:
            Pt.append((y, int(parent[y])))
            y = int(parent[y])
        acc = 0
        for (a, b) in Pt:
            if (a, b) in P:
                sgn = 1
            elif (b, a) in P:
                sgn = -1
            else:
                continue
            rest = [e for e in tedges if set(e) != {a, b}]
            T1 = _component(n, rest, r)
            assert u not in T1
            acc += sgn * int(sum(int(deg[w]) for w in T1))
        f += int(deg[u]) * acc
    return f


def two_forests(g):
    """All 2-forests (spanning forests with exactly two trees) as (T1, T2) vertex
    sets, each forest once; T1 is the tree containing vertex 0."""
    E = [tuple(map(int, e)) for e in g.edges()]
    n = g.n
    out = []
    for comb in itertools.combinations(range(len(E)), n - 2):
        par = list(range(n))

        def find(x):
            while par[x] != x:
                par[x] = par[par[x]]
                x = par[x]
            return x

        ok = True
        for i in comb:
            a, b = E[i]
            ra, rb = find(a), find(b)
            if ra == rb:
                ok = False
                break
            par[ra] = rb
        if ok:
            r0 = find(0)
            T1 = frozenset(v for v in range(n) if find(v) == r0)
            T2 = frozenset(range(n)) - T1
            out.append((T1, T2))
    return out


def K_forest_formula(g, r: int) -> float:
    """Theorem 1: K = 1/(2m |Gamma|) sum_{u != r} d(u) sum_{F in F_{r|u}} vol(T1),
    T1 the tree of F containing r."""
    ntrees = len(spanning_trees(g))
    deg = g.deg
    tot = 0
    for A, B in two_forests(g):
        T1, T2 = (A, B) if r in A else (B, A)
        volT1 = int(sum(int(deg[w]) for w in T1))
        for u in T2:
            tot += int(deg[u]) * volT1
    return tot / (2.0 * g.m * ntrees)


def hoeffding_trees(n: int, m: int, ecc: int, eps: float, delta: float) -> int:
    """Theorem 5 sample size with the two readings: Delta -> ecc(r) (the proof only
    uses the tau0 depth) and kappa >= (n-1)^2/n in place of kappa >= n."""
    kmin = (n - 1) ** 2 / n
    return int(math.ceil(8.0 * m * m * ecc * ecc * math.log(2.0 / delta) / (kmin * kmin * eps * eps)))
