"""The host overlay graph that validates kc_update batches
(paper_2511_16356_gb300/csrc/kc_host_graph.h), compiled with the host C++
compiler and checked against a plain edge-set model with breadth-first
search: edge queries and endpoint connectivity after every insertion and
deletion of long random op sequences, including deletions that disconnect
the graph, re-insertions of deleted base edges and deletions of inserted
edges."""
import ctypes
import os
import shutil
import subprocess
from collections import deque

import numpy as np
import pytest

from paper_2511_16356_gb300 import synth as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2511_16356_gb300", "csrc")

SHIM = r"""
#include "kc_host_graph.h"
extern "C" int hg_run(int64_t n, const int64_t *ro, const int32_t *col, int64_t n_ops,
                      const int32_t *ops, int32_t *out) {
    kc_host::OverlayGraph og(ro, col, n);
    for (int64_t i = 0; i < n_ops; ++i) {
        const int32_t u = ops[3 * i], v = ops[3 * i + 1], op = ops[3 * i + 2];
        const bool present = og.has_edge(u, v);
        out[2 * i] = present ? 1 : 0;
        out[2 * i + 1] = -1;
        if (op == 0 && !present) og.insert(u, v);
        if (op == 1 && present) {
            og.erase(u, v);
            out[2 * i + 1] = og.connected(u, v) ? 1 : 0;
        }
        if (op == 2) out[2 * i + 1] = og.connected(u, v) ? 1 : 0;
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("hostgraph")
    src = d / "shim.cpp"
    src.write_text(SHIM)
    so = d / "shim.so"
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(src), "-o",
                    str(so)], check=True, capture_output=True)
    lib = ctypes.CDLL(str(so))
    lib.hg_run.restype = ctypes.c_int
    lib.hg_run.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                           ctypes.c_void_p, ctypes.c_void_p]
    return lib


def _connected(n, edges, a, b):
    adj = [[] for _ in range(n)]
    for x, y in edges:
        adj[x].append(y)
        adj[y].append(x)
    seen = [False] * n
    seen[a] = True
    q = deque([a])
    while q:
        x = q.popleft()
        if x == b:
            return True
        for y in adj[x]:
            if not seen[y]:
                seen[y] = True
                q.append(y)
    return False


def _run(lib, g, ops):
    ops_arr = np.ascontiguousarray(np.array(ops, dtype=np.int32).reshape(-1, 3))
    out = np.zeros(2 * len(ops), dtype=np.int32)
    lib.hg_run(g.n, g.row_off.ctypes.data, g.col.ctypes.data, len(ops), ops_arr.ctypes.data,
               out.ctypes.data)
    return out.reshape(-1, 2)


def _model(g, ops):
    edges = {(min(int(a), int(b)), max(int(a), int(b))) for a, b in g.edges()}
    want = []
    for u, v, op in ops:
        k = (min(u, v), max(u, v))
        present = k in edges
        conn = -1
        if op == 0 and not present:
            edges.add(k)
        if op == 1 and present:
            edges.discard(k)
            conn = int(_connected(g.n, edges, u, v))
        if op == 2:
            conn = int(_connected(g.n, edges, u, v))
        want.append((int(present), conn))
    return np.array(want, dtype=np.int32)


def _random_ops(g, rng, count):
    edges = sorted({(min(int(a), int(b)), max(int(a), int(b))) for a, b in g.edges()})
    live = set(edges)
    gone = []
    ops = []
    for _ in range(count):
        r = rng.random()
        if r < 0.3 and live:                      # delete a present edge
            e = sorted(live)[int(rng.integers(len(live)))]
            live.discard(e)
            gone.append(e)
            ops.append((e[0], e[1], 1) if rng.random() < 0.5 else (e[1], e[0], 1))
        elif r < 0.45 and gone:                   # re-insert a deleted edge
            e = gone.pop(int(rng.integers(len(gone))))
            live.add(e)
            ops.append((e[1], e[0], 0))
        elif r < 0.7:                             # insert (or fail to insert) a random pair
            a, b = (int(x) for x in rng.choice(g.n, 2, replace=False))
            k = (min(a, b), max(a, b))
            if k not in live:
                live.add(k)
            ops.append((a, b, 0))
        elif r < 0.8:                             # delete a random pair (often absent)
            a, b = (int(x) for x in rng.choice(g.n, 2, replace=False))
            k = (min(a, b), max(a, b))
            if k in live:
                live.discard(k)
                gone.append(k)
            ops.append((a, b, 1))
        else:                                     # query
            a, b = (int(x) for x in rng.choice(g.n, 2, replace=False))
            ops.append((a, b, 2))
    return ops


@pytest.mark.parametrize("make,seed", [
    (lambda: S.er_lcc(60, 0.06, 1), 1), (lambda: S.grid_perturbed(9, 7, 0.2, 2), 2),
    (lambda: S.path(25), 3), (lambda: S.star(12), 4), (lambda: S.complete(8), 5),
    (lambda: S.chung_lu(300, 2.1, 4.0, 6), 6)])
def test_overlay_matches_edge_set_model(shim, make, seed):
    g = make()
    rng = np.random.default_rng(seed)
    ops = _random_ops(g, rng, 600)
    got = _run(shim, g, ops)
    want = _model(g, ops)
    bad = np.nonzero((got != want).any(axis=1))[0]
    assert bad.size == 0, (int(bad[0]), ops[int(bad[0])], got[bad[0]], want[bad[0]])


def test_bridges_of_a_path_and_cycle_edges(shim):
    p = S.path(40)
    got = _run(shim, p, [(i, i + 1, 1) for i in range(0, 39, 3)])
    assert (got[:, 0] == 1).all() and (got[:, 1] == 0).all()  # every path edge is a bridge
    c = S.cycle(40)
    got = _run(shim, c, [(0, 1, 1), (20, 21, 1)])
    assert got[0].tolist() == [1, 1] and got[1].tolist() == [1, 0]  # the second cut splits C40
