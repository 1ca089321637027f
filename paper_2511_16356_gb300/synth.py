"""Seeded synthetic input graphs.

This module only builds inputs: undirected, simple, connected graphs in CSR
form (int64 row offsets, int32 column ids, every row sorted ascending, both
directions of each edge present).  It holds none of the Kemeny-constant
method's arithmetic and is shared by the CPU oracle's tests, the GPU parity
tests and the benchmark.

Workload stand-ins (the paper's SNAP / NetworkRepository graphs are not
available offline; these reproduce their shapes):

* ``er_lcc``       Erdos-Renyi G(n, p), largest connected component
                   (PowerGrid / Hep-th sized static case).
* ``grid_perturbed`` W x H grid with a random spanning tree kept and a fraction
                   of the remaining edges deleted (road-network shaped:
                   degree <= 4, diameter in the thousands).
* ``chung_lu``     Chung-Lu power-law graph with exponent gamma (social shape).
* closed-form families (complete, cycle, star, complete bipartite, path, torus,
  hypercube) and tiny random connected graphs for exact pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_CL_SRC = os.path.join(_HERE, "synth_cl.c")
_CL_LIB = os.path.join(_HERE, "_synth_cl.so")
_cl_lock = threading.Lock()
_cl_handle = None


class Graph:
    """CSR graph: ``row_off`` int64[n+1], ``col`` int32[2m]."""

    def __init__(self, row_off: np.ndarray, col: np.ndarray, name: str = ""):
        self.row_off = np.ascontiguousarray(row_off, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.name = name

    @property
    def n(self) -> int:
        return int(self.row_off.shape[0] - 1)

    @property
    def m(self) -> int:
        return int(self.col.shape[0] // 2)

    @property
    def deg(self) -> np.ndarray:
        return np.diff(self.row_off)

    def neighbors(self, u: int) -> np.ndarray:
        return self.col[self.row_off[u]:self.row_off[u + 1]]

    def edges(self) -> np.ndarray:
        """Undirected edge list (u < v), shape (m, 2)."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), self.deg)
        dst = self.col.astype(np.int64)
        keep = src < dst
        return np.stack([src[keep], dst[keep]], axis=1)

    def __repr__(self) -> str:
        return f"Graph({self.name!r}, n={self.n}, m={self.m})"


def csr_from_edges(n: int, u, v, name: str = "") -> Graph:
    """Symmetric, deduplicated, loop-free CSR with rows sorted ascending."""
    u = np.asarray(u, dtype=np.int64).ravel()
    v = np.asarray(v, dtype=np.int64).ravel()
    keep = u != v
    u, v = u[keep], v[keep]
    a = np.concatenate([u, v])
    b = np.concatenate([v, u])
    key = np.unique(a * np.int64(n) + b)
    src = key // n
    dst = key % n
    counts = np.bincount(src, minlength=n).astype(np.int64)
    row_off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_off[1:])
    return Graph(row_off, dst.astype(np.int32), name)


def components(g: Graph) -> tuple[int, np.ndarray]:
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    a = sp.csr_matrix((np.ones(g.col.shape[0], dtype=np.int8), g.col, g.row_off),
                      shape=(g.n, g.n))
    return connected_components(a, directed=False)


def largest_cc(g: Graph) -> Graph:
    """Induced subgraph on the largest connected component; ids keep their order."""
    ncomp, labels = components(g)
    if ncomp == 1:
        return g
    sizes = np.bincount(labels)
    big = int(np.argmax(sizes))  # ties -> smallest label
    mask = labels == big
    new_id = np.cumsum(mask) - 1
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.deg)
    keep = mask[src]
    s2 = new_id[src[keep]]
    d2 = new_id[g.col[keep].astype(np.int64)]
    n2 = int(mask.sum())
    counts = np.bincount(s2, minlength=n2).astype(np.int64)
    row_off = np.zeros(n2 + 1, dtype=np.int64)
    np.cumsum(counts, out=row_off[1:])
    return Graph(row_off, d2.astype(np.int32), g.name + "/lcc")


def is_connected(g: Graph) -> bool:
    return components(g)[0] == 1


# --------------------------------------------------------------------------
# Closed-form families
# --------------------------------------------------------------------------

def complete(n: int) -> Graph:
    iu = np.triu_indices(n, 1)
    return csr_from_edges(n, iu[0], iu[1], f"K{n}")


def cycle(n: int) -> Graph:
    i = np.arange(n)
    return csr_from_edges(n, i, (i + 1) % n, f"C{n}")


def path(n: int) -> Graph:
    i = np.arange(n - 1)
    return csr_from_edges(n, i, i + 1, f"P{n}")


def star(n: int) -> Graph:
    """K_{1,n-1} with centre 0."""
    i = np.arange(1, n)
    return csr_from_edges(n, np.zeros(n - 1, dtype=np.int64), i, f"S{n}")


def complete_bipartite(a: int, b: int) -> Graph:
    uu, vv = np.meshgrid(np.arange(a), a + np.arange(b), indexing="ij")
    return csr_from_edges(a + b, uu.ravel(), vv.ravel(), f"K{a},{b}")


def grid(w: int, h: int) -> Graph:
    """w x h grid, vertex id y * w + x."""
    ids = np.arange(w * h).reshape(h, w)
    hu, hv = ids[:, :-1].ravel(), ids[:, 1:].ravel()
    vu, vv = ids[:-1, :].ravel(), ids[1:, :].ravel()
    return csr_from_edges(w * h, np.concatenate([hu, vu]), np.concatenate([hv, vv]),
                          f"grid{w}x{h}")


def torus(a: int, b: int) -> Graph:
    """a x b discrete torus (a, b >= 3 so that it is simple and 4-regular)."""
    ids = np.arange(a * b).reshape(b, a)
    hu, hv = ids.ravel(), np.roll(ids, -1, axis=1).ravel()
    vu, vv = ids.ravel(), np.roll(ids, -1, axis=0).ravel()
    return csr_from_edges(a * b, np.concatenate([hu, vu]), np.concatenate([hv, vv]),
                          f"torus{a}x{b}")


def hypercube(k: int) -> Graph:
    n = 1 << k
    i = np.arange(n, dtype=np.int64)
    us, vs = [], []
    for bit in range(k):
        j = i ^ (1 << bit)
        keep = i < j
        us.append(i[keep])
        vs.append(j[keep])
    return csr_from_edges(n, np.concatenate(us), np.concatenate(vs), f"Q{k}")


def random_connected(n: int, p: float, seed: int) -> Graph:
    """G(n, p) conditioned on being connected (rejection on the seed stream)."""
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(n, 1)
    for _ in range(10000):
        keep = rng.random(iu[0].shape[0]) < p
        g = csr_from_edges(n, iu[0][keep], iu[1][keep], f"rc{n}_{seed}")
        if g.n == n and np.all(g.deg > 0) and is_connected(g):
            return g
    raise RuntimeError("could not draw a connected graph")


# --------------------------------------------------------------------------
# Workload stand-ins
# --------------------------------------------------------------------------

def er_lcc(n: int, p: float, seed: int) -> Graph:
    rng = np.random.default_rng(seed)
    if n <= 5000:
        iu = np.triu_indices(n, 1)
        keep = rng.random(iu[0].shape[0]) < p
        g = csr_from_edges(n, iu[0][keep], iu[1][keep], f"er{n}_{seed}")
        return largest_cc(g)
    # large n: successes of the pair sequence (i < j, row-major) by geometric gaps
    npairs = n * (n - 1) // 2
    want = int(npairs * p + 10 * np.sqrt(npairs * p) + 100)
    gaps = rng.geometric(p, size=want).astype(np.int64)
    idx = np.cumsum(gaps) - 1
    idx = idx[idx < npairs]
    row_start = np.concatenate([[0], np.cumsum(np.arange(n - 1, 0, -1, dtype=np.int64))])
    i = np.searchsorted(row_start, idx, side="right") - 1
    j = i + 1 + (idx - row_start[i])
    g = csr_from_edges(n, i, j, f"er{n}_{seed}")
    return largest_cc(g)


def grid_perturbed(w: int, h: int, delete_frac: float, seed: int) -> Graph:
    """w x h grid; a random spanning tree (minimum spanning tree under i.i.d.
    uniform edge weights) is kept and round(delete_frac * m0) of the other
    edges, chosen uniformly, are deleted, so the result stays connected."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import minimum_spanning_tree

    rng = np.random.default_rng(seed)
    ids = np.arange(w * h, dtype=np.int64).reshape(h, w)
    eu = np.concatenate([ids[:, :-1].ravel(), ids[:-1, :].ravel()])
    ev = np.concatenate([ids[:, 1:].ravel(), ids[1:, :].ravel()])
    m0 = eu.shape[0]
    n = w * h
    wts = 1.0 + rng.random(m0)
    t = minimum_spanning_tree(coo_matrix((wts, (eu, ev)), shape=(n, n)).tocsr()).tocoo()
    tu = np.minimum(t.row, t.col).astype(np.int64)
    tv = np.maximum(t.row, t.col).astype(np.int64)
    in_tree = np.zeros(m0, dtype=bool)
    # edge index lookup: key -> index
    key = eu * n + ev
    order = np.argsort(key)
    pos = np.searchsorted(key[order], tu * n + tv)
    in_tree[order[pos]] = True
    assert in_tree.sum() == n - 1
    non_tree = np.flatnonzero(~in_tree)
    k = int(round(delete_frac * m0))
    k = min(k, non_tree.shape[0])
    drop = rng.choice(non_tree, size=k, replace=False)
    keep = np.ones(m0, dtype=bool)
    keep[drop] = False
    return csr_from_edges(n, eu[keep], ev[keep], f"grid{w}x{h}-{delete_frac:g}_{seed}")


def _cl_lib():
    global _cl_handle
    with _cl_lock:
        if _cl_handle is None:
            if (not os.path.exists(_CL_LIB)
                    or os.path.getmtime(_CL_LIB) < os.path.getmtime(_CL_SRC)):
                tmp = _CL_LIB + f".{os.getpid()}.tmp"
                subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp,
                                       _CL_SRC, "-lm"])
                os.replace(tmp, _CL_LIB)
            lib = ctypes.CDLL(_CL_LIB)
            lib.synth_chung_lu.restype = ctypes.c_int64
            lib.synth_chung_lu.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_uint64,
                                           ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
            _cl_handle = lib
        return _cl_handle


def chung_lu_weights(n: int, gamma: float, mean_deg: float) -> np.ndarray:
    """w_i = c (i + i0)^(-1/(gamma-1)), mean mean_deg, largest weight sqrt(n*mean_deg)
    (so that w_i w_j / W <= 1 for every pair)."""
    a = 1.0 / (gamma - 1.0)
    i = np.arange(n, dtype=np.float64)
    target = np.sqrt(n / mean_deg)  # w_0 / mean(w)

    def ratio(i0):
        x = (i + i0) ** (-a)
        return x[0] / x.mean()

    lo, hi = 1e-6, float(n)
    for _ in range(200):
        mid = np.sqrt(lo * hi)
        if ratio(mid) > target:
            lo = mid
        else:
            hi = mid
    x = (i + hi) ** (-a)
    return x * (mean_deg / x.mean())


def chung_lu(n: int, gamma: float, mean_deg: float, seed: int, lcc: bool = True) -> Graph:
    w = chung_lu_weights(n, gamma, mean_deg)
    lib = _cl_lib()
    cap = int(n * mean_deg * 0.75) + 1024
    while True:
        eu = np.empty(cap, dtype=np.int32)
        ev = np.empty(cap, dtype=np.int32)
        m = lib.synth_chung_lu(n, w.ctypes.data, seed, cap, eu.ctypes.data, ev.ctypes.data)
        if m >= 0:
            break
        cap *= 2
    g = csr_from_edges(n, eu[:m], ev[:m], f"cl{n}_g{gamma:g}_d{mean_deg:g}_{seed}")
    return largest_cc(g) if lcc else g


# --------------------------------------------------------------------------
# Named workloads (the configurations benchmarked and parity-tested)
# --------------------------------------------------------------------------

WORKLOADS = {
    "er2000": "Erdos-Renyi G(2000, 8/1999), seed 0, largest connected component",
    "grid1000": "1000x1000 grid, random spanning tree kept, 25% of all edges deleted "
                "among the rest, seed 1 (n = 1,000,000, m = 1,498,500)",
    "cl4m": "Chung-Lu gamma=2.1, n=4,000,000, mean degree 17, seed 2, largest component",
}


def workload(name: str) -> Graph:
    if name == "er2000":
        return er_lcc(2000, 8.0 / 1999.0, 0)
    if name == "grid1000":
        return grid_perturbed(1000, 1000, 0.25, 1)
    if name == "cl4m":
        return chung_lu(4_000_000, 2.1, 17.0, 2)
    if name.startswith("grid") and "x" in name:
        w, h = name[4:].split("x")
        return grid_perturbed(int(w), int(h), 0.25, 1)
    if name.startswith("er") and name[2:].isdigit():
        n = int(name[2:])
        return er_lcc(n, 8.0 / (n - 1), 0)
    if name.startswith("cl") and name[2:].isdigit():
        return chung_lu(int(name[2:]), 2.1, 17.0, 2)
    raise KeyError(name)
