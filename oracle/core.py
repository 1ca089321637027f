"""ctypes front end of the plain-C oracle core (kc_oracle.c).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

__all__ = [
    "build_oracle", "lib", "philox4x32_10", "bounded", "root", "root_smallest_id", "bfs_tree", "dfs_tree",
    "Tau0",
    "tau0", "wilson", "traverse", "f_naive", "f_alg1", "TreeOut", "tree",
    "sample_batch", "num_threads", "STEP_CAP_DEFAULT", "cond_wilson", "select", "link_cut",
    "cut_link",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "kc_oracle.c"), os.path.join(_HERE, "kc_oracle_dyn.c")]
_LIB = os.path.join(_HERE, "_kc_oracle.so")
_lock = threading.Lock()
_handle = None

STEP_CAP_DEFAULT = 1 << 62

_i64p = ctypes.c_void_p


def build_oracle(force: bool = False) -> str:
    """Compile the oracle C sources with gcc (-O2, OpenMP across trees)."""
    srcs = [s for s in _SRC if os.path.exists(s)]
    stale = force or not os.path.exists(_LIB) or any(
        os.path.getmtime(_LIB) < os.path.getmtime(s) for s in srcs)
    if stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, *srcs])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _handle
    with _lock:
        if _handle is None:
            build_oracle()
            L = ctypes.CDLL(_LIB)
            c_i64, c_i32, c_u32, c_u64, vp = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32,
                                              ctypes.c_uint64, ctypes.c_void_p)
            L.orc_philox4x32_10.argtypes = [vp, vp, vp]
            L.orc_philox4x32_10.restype = None
            L.orc_bounded.argtypes = [c_u64, c_u32, c_u32, c_u32, c_u32, c_u32]
            L.orc_bounded.restype = c_u32
            L.orc_root.argtypes = [c_i64, vp]
            L.orc_root.restype = c_i32
            L.orc_root_central.argtypes = [c_i64, vp, vp]
            L.orc_root_central.restype = c_i32
            L.orc_bfs_tree.argtypes = [c_i64, vp, vp, c_i32, vp, vp]
            L.orc_bfs_tree.restype = c_i32
            L.orc_dfs_tree.argtypes = [c_i64, vp, vp, c_i32, vp, vp]
            L.orc_dfs_tree.restype = c_i32
            L.orc_wilson.argtypes = [c_i64, vp, vp, c_i32, c_u64, c_u32, vp, vp, vp, c_i64]
            L.orc_wilson.restype = ctypes.c_int
            L.orc_traverse.argtypes = [c_i64, vp, vp, c_i32, vp, vp, vp, vp, vp]
            L.orc_traverse.restype = ctypes.c_int
            L.orc_f_naive.argtypes = [c_i64, vp, c_i32, vp, vp, vp]
            L.orc_f_naive.restype = c_i64
            L.orc_f_alg1.argtypes = [c_i64, vp, c_i32, vp, vp, vp, vp, vp]
            L.orc_f_alg1.restype = c_i64
            L.orc_sample_batch.argtypes = [c_i64, vp, vp, c_i32, vp, vp, vp, c_u64, c_u32, c_i64,
                                           ctypes.c_int, ctypes.c_int, c_i64, vp, vp]
            L.orc_sample_batch.restype = ctypes.c_int
            L.orc_cond_wilson.argtypes = [c_i64, vp, vp, c_i32, c_i32, c_i32, c_u64, c_u32, vp,
                                          vp, c_i64]
            L.orc_cond_wilson.restype = ctypes.c_int
            L.orc_select.argtypes = [c_u64, c_u32, c_i64, c_i64, vp]
            L.orc_select.restype = None
            for fn in (L.orc_link_cut, L.orc_cut_link):
                fn.argtypes = [c_i64, vp, vp, vp, c_i32, c_i32, c_i32, c_u64, c_u32, c_u32, c_i64,
                               vp, vp, vp]
                fn.restype = ctypes.c_int
            L.orc_num_threads.argtypes = []
            L.orc_num_threads.restype = ctypes.c_int
            _handle = L
        return _handle


def _p(a: np.ndarray):
    return a.ctypes.data


def num_threads() -> int:
    return int(lib().orc_num_threads())


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def bounded(seed: int, c0: int, c1: int, c2: int, tag: int, s: int) -> int:
    return int(lib().orc_bounded(seed, c0, c1, c2, tag, s))


def root(g) -> int:
    """Highest degree, ties broken towards the double-sweep centre, then smallest id."""
    return int(lib().orc_root_central(g.n, _p(g.row_off), _p(g.col)))


def root_smallest_id(g) -> int:
    """Highest degree, smallest id among ties."""
    return int(lib().orc_root(g.n, _p(g.row_off)))


def bfs_tree(g, r: int):
    p0 = np.empty(g.n, dtype=np.int32)
    level = np.empty(g.n, dtype=np.int32)
    ecc = lib().orc_bfs_tree(g.n, _p(g.row_off), _p(g.col), r, _p(p0), _p(level))
    return p0, level, int(ecc)


def dfs_tree(g, r: int):
    """Depth-first spanning tree from r, rows scanned in ascending id (Exp-II)."""
    p0 = np.empty(g.n, dtype=np.int32)
    level = np.empty(g.n, dtype=np.int32)
    deepest = lib().orc_dfs_tree(g.n, _p(g.row_off), _p(g.col), r, _p(p0), _p(level))
    return p0, level, int(deepest)


class TreeOut:
    """Per-tree outputs: parent, depth, size, vol, DFN in/out, steps, f."""

    def __init__(self, n):
        self.parent = np.empty(n, dtype=np.int32)
        self.depth = np.empty(n, dtype=np.int32)
        self.size = np.empty(n, dtype=np.int32)
        self.vol = np.empty(n, dtype=np.int64)
        self.din = np.empty(n, dtype=np.int32)
        self.dout = np.empty(n, dtype=np.int32)
        self.steps = 0
        self.f = 0


class Tau0:
    """Root r, path tree tau0 (parent p0, DFN in0/out0, volumes) and its depth
    `ecc`.  kind: "bfs" (Algorithm 1; depth = ecc(r)), "dfs" or "wilson" (the
    other path selections of Exp-II; "wilson" is the uniform tree of sample id 0
    under `seed`).  Theorem 4 holds for any fixed spanning tree tau0."""

    def __init__(self, g, r=None, kind: str = "bfs", seed: int = 0):
        self.r = root(g) if r is None else int(r)
        self.kind = kind
        if kind == "bfs":
            self.p0, self.level, self.ecc = bfs_tree(g, self.r)
        elif kind == "dfs":
            self.p0, self.level, self.ecc = dfs_tree(g, self.r)
        elif kind == "wilson":
            parent, _ = wilson(g, self.r, seed, 0)
            self.p0 = parent.astype(np.int32)
            t = traverse(g, self.r, self.p0)
            self.level = t.depth.copy()
            self.ecc = int(self.level.max())
        else:
            raise ValueError(kind)
        if self.ecc < 0:
            raise ValueError("graph is disconnected")
        t = TreeOut(g.n)
        rc = lib().orc_traverse(g.n, _p(g.row_off), _p(self.p0), self.r, _p(t.depth),
                                _p(t.size), _p(t.vol), _p(t.din), _p(t.dout))
        assert rc == 0
        self.in0, self.out0, self.vol0, self.size0 = t.din, t.dout, t.vol, t.size


def tau0(g, r=None, kind: str = "bfs", seed: int = 0) -> Tau0:
    return Tau0(g, r, kind, seed)


def wilson(g, r: int, seed: int, sample: int, order=None, cap: int = STEP_CAP_DEFAULT):
    parent = np.empty(g.n, dtype=np.int32)
    steps = np.zeros(1, dtype=np.int64)
    o = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    rc = lib().orc_wilson(g.n, _p(g.row_off), _p(g.col), r, seed, sample,
                          None if o is None else _p(o), _p(parent), _p(steps), cap)
    if rc:
        raise RuntimeError("step cap exceeded")
    return parent, int(steps[0])


def traverse(g, r: int, parent: np.ndarray) -> TreeOut:
    t = TreeOut(g.n)
    t.parent[:] = parent
    rc = lib().orc_traverse(g.n, _p(g.row_off), _p(t.parent), r, _p(t.depth), _p(t.size),
                            _p(t.vol), _p(t.din), _p(t.dout))
    if rc:
        raise ValueError("parent array is not a spanning tree rooted at r")
    return t


def f_naive(g, t0: Tau0, parent: np.ndarray, vol: np.ndarray) -> int:
    return int(lib().orc_f_naive(g.n, _p(g.row_off), t0.r,
                                 _p(np.ascontiguousarray(parent, dtype=np.int32)),
                                 _p(np.ascontiguousarray(vol, dtype=np.int64)), _p(t0.p0)))


def f_alg1(g, t0: Tau0, parent: np.ndarray, vol: np.ndarray) -> int:
    return int(lib().orc_f_alg1(g.n, _p(g.row_off), t0.r,
                                _p(np.ascontiguousarray(parent, dtype=np.int32)),
                                _p(np.ascontiguousarray(vol, dtype=np.int64)), _p(t0.p0),
                                _p(t0.in0), _p(t0.out0)))


def tree(g, t0: Tau0, seed: int, sample: int, method: str = "alg1", order=None) -> TreeOut:
    """Everything the sampler computes for one sample id."""
    parent, steps = wilson(g, t0.r, seed, sample, order)
    t = traverse(g, t0.r, parent)
    t.steps = steps
    t.f = f_alg1(g, t0, parent, t.vol) if method == "alg1" else f_naive(g, t0, parent, t.vol)
    return t


def sample_batch(g, t0: Tau0, seed: int, id0: int, count: int, method: str = "alg1",
                 threads: int = 0, cap: int = STEP_CAP_DEFAULT):
    """f and step counts for sample ids [id0, id0 + count)."""
    f = np.zeros(count, dtype=np.int64)
    steps = np.zeros(count, dtype=np.int64)
    rc = lib().orc_sample_batch(g.n, _p(g.row_off), _p(g.col), t0.r, _p(t0.p0), _p(t0.in0),
                                _p(t0.out0), seed, id0, count, 1 if method == "naive" else 0,
                                threads, cap, _p(f), _p(steps))
    if rc:
        raise RuntimeError("step cap exceeded")
    return f, steps


def cond_wilson(g, u: int, v: int, r: int, seed: int, sample: int, cap: int = STEP_CAP_DEFAULT):
    """Uniform spanning tree of g conditioned on containing (u, v), rooted at r."""
    parent = np.empty(g.n, dtype=np.int32)
    steps = np.zeros(1, dtype=np.int64)
    rc = lib().orc_cond_wilson(g.n, _p(g.row_off), _p(g.col), u, v, r, seed, sample, _p(parent),
                               _p(steps), cap)
    if rc:
        raise RuntimeError("step cap exceeded")
    return parent, int(steps[0])


def select(seed: int, seq: int, N: int, k: int) -> np.ndarray:
    out = np.empty(max(k, 1), dtype=np.int64)
    lib().orc_select(seed, seq, N, k, _p(out))
    return out[:k]


def _transform(fn, g, parent, r, u, v, seed, seq, pool_idx, k_force):
    out = np.empty(g.n, dtype=np.int32)
    d_old = np.zeros(1, dtype=np.int64)
    d_new = np.zeros(1, dtype=np.int64)
    fn(g.n, _p(g.row_off), _p(g.col), _p(np.ascontiguousarray(parent, dtype=np.int32)), r, u, v,
       seed, seq, pool_idx, k_force, _p(out), _p(d_old), _p(d_new))
    return out, int(d_old[0]), int(d_new[0])


def link_cut(g, parent, r, u, v, seed=0, seq=0, pool_idx=0, k_force=-1):
    """link-cut of a tree of g - (u,v) into a tree of g (which contains (u,v))."""
    return _transform(lib().orc_link_cut, g, parent, r, u, v, seed, seq, pool_idx, k_force)


def cut_link(g, parent, r, u, v, seed=0, seq=0, pool_idx=0, k_force=-1):
    """cut-link of a tree containing (u,v) into a tree of g (from which (u,v) is removed)."""
    return _transform(lib().orc_cut_link, g, parent, r, u, v, seed, seq, pool_idx, k_force)
