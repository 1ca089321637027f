"""The decomposition behind the segmented BIT evaluation of f (Algorithm 1 over
the tau preorder, split into segments), checked on the CPU without the CUDA
path.

Algorithm 1 visits the vertices of tau in preorder; at each vertex it first
undoes the range adds of the stacked ancestors whose subtree has ended, then
applies the vertex's own range add (over a tau0-DFN interval, Theorem 4) and
reads Q(v) at in0(v).  The segmented evaluation starts a segment at position
lo with the stack holding the strict tau-ancestors of the vertex at lo that add
a range (root side first) and the range array holding the sum of their adds,
then runs the same steps over [lo, hi).  This test replays that in plain
Python with a difference array instead of a Fenwick array: for every tree and
every split the sum of the segments' d(v) Q(v) must equal the oracle's f, and
so must the unsplit sweep.  Dropping the initial ancestors, or stacking them in
the wrong order, makes the split sums differ."""
import numpy as np
import pytest

import oracle as O
from paper_2511_16356_gb300 import synth as S


def _range_entries(g, t0, tr):
    """Per vertex x != r: (l, r, val) of its range add, or None (Theorem 4:
    forward when p(x) = p0(x), reverse when p0(p(x)) = x)."""
    twom = 2 * g.m
    out = [None] * g.n
    for x in range(g.n):
        if x == t0.r:
            continue
        par = int(tr.parent[x])
        if int(t0.p0[x]) == par:
            out[x] = (int(t0.in0[x]), int(t0.out0[x]), twom - int(tr.vol[x]))
        elif par != t0.r and int(t0.p0[par]) == x:
            out[x] = (int(t0.in0[par]), int(t0.out0[par]), int(tr.vol[x]) - twom)
    return out


def _sweep(g, t0, tr, order, entries, lo, hi, start_stack):
    """Algorithm 1's steps over preorder positions [lo, hi) from the given
    stack (a list of (end, l, r, val), deepest last); returns sum d(v) Q(v)."""
    deg = np.diff(g.row_off)
    diff = np.zeros(g.n + 1, dtype=np.int64)
    stack = []
    for e in start_stack:
        stack.append(e)
        diff[e[1]] += e[3]
        diff[e[2] + 1] -= e[3]
    total = 0
    for i in range(lo, hi):
        v = int(order[i])
        while stack and stack[-1][0] < i:
            _, l, r, val = stack.pop()
            diff[l] -= val
            diff[r + 1] += val
        if entries[v] is not None:
            l, r, val = entries[v]
            stack.append((i + int(tr.size[v]) - 1, l, r, val))
            diff[l] += val
            diff[r + 1] -= val
        q = int(diff[: int(t0.in0[v]) + 1].sum())
        total += int(deg[v]) * q
    return total


def _start_stack(t0, tr, order, entries, lo):
    """Strict tau-ancestors of the vertex at position lo that add a range,
    root side first, as stack entries."""
    chain = []
    x = int(tr.parent[int(order[lo])])
    while x >= 0 and x != t0.r:
        if entries[x] is not None:
            l, r, val = entries[x]
            chain.append((int(tr.din[x]) + int(tr.size[x]) - 1, l, r, val))
        x = int(tr.parent[x])
    return chain[::-1]


GRAPHS = {
    "grid17x13": lambda: S.grid_perturbed(17, 13, 0.25, 3),
    "er300": lambda: S.er_lcc(300, 0.02, 7),
    "path33": lambda: S.path(33),
    "star9": lambda: S.star(9),
    "K3,5": lambda: S.complete_bipartite(3, 5),
    "cycle40": lambda: S.cycle(40),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_split_sweeps_sum_to_f(name):
    g = GRAPHS[name]()
    t0 = O.tau0(g)
    for sample in range(4):
        tr = O.tree(g, t0, 77, sample)
        order = np.argsort(tr.din, kind="stable")
        assert np.array_equal(tr.din[order], np.arange(g.n))  # din is a preorder
        entries = _range_entries(g, t0, tr)
        assert _sweep(g, t0, tr, order, entries, 0, g.n, []) == tr.f
        for k in (2, 3, 7, g.n, g.n + 5):
            total = 0
            for j in range(k):
                lo, hi = j * g.n // k, (j + 1) * g.n // k
                if lo == hi:
                    continue
                start = _start_stack(t0, tr, order, entries, lo) if lo > 0 else []
                total += _sweep(g, t0, tr, order, entries, lo, hi, start)
            assert total == tr.f, (name, sample, k)


def test_split_without_the_ancestors_differs():
    """The rebuilt state matters: starting each segment from an empty stack
    gives a different sum on a tree with deep forward entries."""
    g = GRAPHS["grid17x13"]()
    t0 = O.tau0(g)
    tr = O.tree(g, t0, 77, 0)
    order = np.argsort(tr.din, kind="stable")
    entries = _range_entries(g, t0, tr)
    k = 5
    wrong = sum(_sweep(g, t0, tr, order, entries, j * g.n // k, (j + 1) * g.n // k, [])
                for j in range(k))
    assert wrong != tr.f
