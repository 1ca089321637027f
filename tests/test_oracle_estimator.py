"""Pins of the oracle's per-tree estimator f(tau).

* Unbiasedness (Theorem 3): the uniform average of f/(2m) over ALL spanning
  trees (enumerated, count checked by Kirchhoff) equals exact K to 1e-12.
* Three independent routes agree per tree: the literal Definition 1 /
  Theorem 3 construction (explicit 2-forests), the naive path comparison and
  Algorithm 1 (DFS + BIT with the corrected undo).
* f(tau0) has the closed form sum_w (2m - vol0(w)) vol0(w).
* The worked triangle example of Sec. 3.1 (golden file).
* Algorithm 1 with the reverse-case undo exactly as printed is wrong on some
  trees (erratum), while the corrected one matches the naive route.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2511_16356_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

SMALL = {
    "K3": lambda: S.complete(3),
    "K5": lambda: S.complete(5),
    "C6": lambda: S.cycle(6),
    "K2,3": lambda: S.complete_bipartite(2, 3),
    "grid3x3": lambda: S.grid(3, 3),
    "rc7": lambda: S.random_connected(7, 0.5, 3),
    "rc8": lambda: S.random_connected(8, 0.4, 21),
    "torus3x3": lambda: S.torus(3, 3),
}


def _all_f(g, t0, literal=True):
    rows = []
    for T in O.spanning_trees(g):
        par = O.orient(g.n, T, t0.r)
        t = O.traverse(g, t0.r, par)
        a = O.f_alg1(g, t0, par, t.vol)
        b = O.f_naive(g, t0, par, t.vol)
        c = O.f_literal(g, t0.r, t0.p0, par) if literal else b
        rows.append((a, b, c))
    return np.array(rows, dtype=np.int64)


@pytest.mark.parametrize("name", list(SMALL))
def test_unbiased_by_enumeration(name):
    g = SMALL[name]()
    t0 = O.tau0(g)
    F = _all_f(g, t0, literal=g.m <= 12)
    assert np.array_equal(F[:, 0], F[:, 1])
    assert np.array_equal(F[:, 0], F[:, 2])
    k_hat = F[:, 0].mean() / (2 * g.m)
    assert k_hat == pytest.approx(O.K_dense(g), rel=1e-12)


@pytest.mark.parametrize("r", [0, 2, 4])
def test_unbiased_for_any_root_and_any_tau0(r):
    """Theorem 4 holds for an arbitrary fixed spanning tree tau0 (not only BFS)."""
    g = S.random_connected(7, 0.5, 3)
    t0 = O.tau0(g, r)
    trees = O.spanning_trees(g)
    # replace tau0 by a non-BFS spanning tree: the last enumerated tree
    alt = O.orient(g.n, trees[-1], r)
    t0.p0 = alt
    tt = O.traverse(g, r, alt)
    t0.in0, t0.out0 = tt.din, tt.dout
    fs = []
    for T in trees:
        par = O.orient(g.n, T, r)
        t = O.traverse(g, r, par)
        a = O.f_alg1(g, t0, par, t.vol)
        assert a == O.f_naive(g, t0, par, t.vol)
        fs.append(a)
    assert np.mean(fs) / (2 * g.m) == pytest.approx(O.K_dense(g), rel=1e-12)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_alg1_equals_naive_on_sampled_trees(seed):
    g = S.er_lcc(300, 0.02, seed)
    t0 = O.tau0(g)
    for k in range(6):
        t = O.tree(g, t0, seed, k)
        assert t.f == O.f_naive(g, t0, t.parent, t.vol)


def test_f_of_tau0_closed_form():
    g = S.er_lcc(200, 0.04, 5)
    t0 = O.tau0(g)
    t = O.traverse(g, t0.r, t0.p0)
    twom = 2 * g.m
    want = int(sum((twom - int(t.vol[w])) * int(t.vol[w]) for w in range(g.n) if w != t0.r))
    assert O.f_alg1(g, t0, t0.p0, t.vol) == want
    assert O.f_naive(g, t0, t0.p0, t.vol) == want


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if not line:
            continue
        k, v = line.split()[:2]
        out[k] = int(v)
    return out


def test_triangle_worked_example():
    gold = _golden("k3_triangle.txt")
    g = S.complete(3)
    v1, v2, v3 = 0, 1, 2
    r = v1
    p0 = np.array([-1, v3, v1], dtype=np.int32)  # P_{v2}: v2 -> v3 -> v1
    tau1 = np.array([-1, v3, v1], dtype=np.int32)  # path v2 -> v3 -> v1
    tau3 = np.array([-1, v1, v1], dtype=np.int32)  # direct v2 -> v1, contains (v1, v3)
    tau2 = np.array([-1, v1, v2], dtype=np.int32)  # the remaining tree
    assert len(O.spanning_trees(g)) == gold["n_spanning_trees"]
    d = g.deg
    # f restricted to u = v2 is d(v2) * (sum of vol(T1) over the mapped forests)
    f1 = O.f_literal(g, r, p0, tau1, u_only=v2)
    # the two forests F3 = tau1 \ (v2,v3) (T1 = {v1, v3}) and F1 = tau1 \ (v3,v1) (T1 = {v1})
    assert f1 == d[v2] * ((d[v1] + d[v3]) + gold["F1_vol_T1"])
    assert gold["tau1_forward_forest_count_u_v2"] == 2
    assert O.f_literal(g, r, p0, tau3, u_only=v2) == 0 and gold["tau3_forest_count_u_v2"] == 0
    assert O.f_literal(g, r, p0, tau2, u_only=v2) == 0 and gold["tau2_forest_count_u_v2"] == 0
    # F_{v2|v1}: two-forests separating v1 and v2
    sep = [F for F in O.two_forests(g) if (v1 in F[0]) != (v2 in F[0])]
    assert len(sep) == gold["F_v2_given_v1_count"]
    vols = sorted(int(sum(d[w] for w in (A if v1 in A else B))) for A, B in sep)
    assert gold["F1_vol_T1"] in vols
    # and the estimator over the three trees recovers K(K3) = 4/3 for this non-BFS tau0
    t0 = O.tau0(g, r)
    t0.p0 = p0
    tt = O.traverse(g, r, p0)
    t0.in0, t0.out0 = tt.din, tt.dout
    fs = [O.f_alg1(g, t0, t, O.traverse(g, r, t).vol) for t in (tau1, tau2, tau3)]
    assert np.mean(fs) / (2 * g.m) == pytest.approx(4.0 / 3.0, rel=1e-15)


def _alg1_as_printed(g, t0, parent, vol):
    """Algorithm 1 with the reverse-case undo exactly as printed (adds vol - 2m again
    instead of negating the reverse-case add)."""
    n = g.n
    twom = 2 * g.m
    deg = g.deg
    bit = np.zeros(n + 2, dtype=np.int64)

    def add(i, val):
        i += 1
        while i <= n:
            bit[i] += val
            i += i & -i

    def radd(l, r, val):
        add(l, val)
        if r + 1 < n:
            add(r + 1, -val)

    def q(i):
        i += 1
        s = 0
        while i > 0:
            s += bit[i]
            i -= i & -i
        return int(s)

    children = [[] for _ in range(n)]
    for v in range(n):
        if v != t0.r:
            children[parent[v]].append(v)
    f = 0

    def dfs(v):
        nonlocal f
        p = parent[v] if v != t0.r else -1
        kind = 0
        if v != t0.r:
            if t0.p0[v] == p:
                radd(t0.in0[v], t0.out0[v], twom - vol[v]); kind = 1
            elif p != t0.r and t0.p0[p] == v:
                radd(t0.in0[p], t0.out0[p], vol[v] - twom); kind = 2
        f += int(deg[v]) * q(t0.in0[v])
        for c in children[v]:
            dfs(c)
        if kind == 1:
            radd(t0.in0[v], t0.out0[v], vol[v] - twom)
        elif kind == 2:
            radd(t0.in0[p], t0.out0[p], vol[v] - twom)  # as printed

    dfs(t0.r)
    return f


def test_printed_undo_is_wrong_corrected_is_right():
    wrong = 0
    total = 0
    for seed in range(3):
        g = S.er_lcc(100, 0.05, 100 + seed)
        t0 = O.tau0(g)
        for k in range(20):
            t = O.tree(g, t0, seed, k)
            naive = O.f_naive(g, t0, t.parent, t.vol)
            assert t.f == naive
            wrong += _alg1_as_printed(g, t0, t.parent, t.vol) != naive
            total += 1
    assert wrong > total // 2, "the printed reverse-case undo should disagree on most trees"


def _dfs_recursive(g, r):
    """Textbook recursive DFS (rows in ascending id), written independently of
    the oracle's explicit-stack version."""
    import sys

    sys.setrecursionlimit(max(10000, 4 * g.n))
    parent = [-2] * g.n
    depth = [0] * g.n

    def visit(u):
        for e in range(int(g.row_off[u]), int(g.row_off[u + 1])):
            w = int(g.col[e])
            if parent[w] == -2:
                parent[w] = u
                depth[w] = depth[u] + 1
                visit(w)

    parent[r] = -1
    visit(r)
    return np.array(parent, dtype=np.int32), np.array(depth, dtype=np.int32)


@pytest.mark.parametrize("gname", ["grid6x5", "er60", "K7", "star9"])
def test_dfs_path_tree_matches_recursive_dfs(gname):
    g = {"grid6x5": lambda: S.grid(6, 5), "er60": lambda: S.er_lcc(60, 0.1, 3),
         "K7": lambda: S.complete(7), "star9": lambda: S.star(9)}[gname]()
    t0 = O.tau0(g, kind="dfs")
    p, d = _dfs_recursive(g, t0.r)
    assert np.array_equal(t0.p0, p) and np.array_equal(t0.level, d)
    assert t0.ecc == d.max()


@pytest.mark.parametrize("kind", ["dfs", "wilson"])
@pytest.mark.parametrize("name", ["K4", "grid3x3", "rc7"])
def test_unbiased_for_dfs_and_wilson_path_trees(name, kind):
    """Exp-II's other path selections: for a DFS tree or a Wilson tree as tau0,
    the uniform average of f/(2m) over every spanning tree is still exactly K
    (Theorem 4 holds for any fixed tau0), and Algorithm 1 equals the naive
    form tree by tree."""
    g = {"K4": lambda: S.complete(4), "grid3x3": lambda: S.grid(3, 3),
         "rc7": lambda: S.random_connected(7, 0.5, 2)}[name]()
    t0 = O.tau0(g, kind=kind, seed=9)
    fs = []
    for T in O.spanning_trees(g):
        par = O.orient(g.n, T, t0.r)
        t = O.traverse(g, t0.r, par)
        a = O.f_alg1(g, t0, par, t.vol)
        assert a == O.f_naive(g, t0, par, t.vol)
        fs.append(a)
    assert np.mean(fs) / (2 * g.m) == pytest.approx(O.K_dense(g), rel=1e-12)


@pytest.mark.parametrize("gname", ["grid7x5", "er80", "cl400"])
def test_path_trees_against_networkx(gname):
    """BFS levels of tau0 equal networkx shortest-path lengths from the root,
    and the DFS path tree equals networkx's depth-first tree (adjacency in
    ascending id)."""
    nx = pytest.importorskip("networkx")
    g = {"grid7x5": lambda: S.grid(7, 5), "er80": lambda: S.er_lcc(80, 0.08, 2),
         "cl400": lambda: S.chung_lu(400, 2.1, 6.0, 3)}[gname]()
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    src = np.repeat(np.arange(g.n), g.deg)
    G.add_edges_from((int(a), int(b)) for a, b in zip(src, g.col) if a < b)
    bfs = O.tau0(g)
    dist = nx.single_source_shortest_path_length(G, bfs.r)
    assert all(bfs.level[v] == dist[v] for v in range(g.n))
    dfs = O.tau0(g, kind="dfs")
    pred = nx.dfs_predecessors(G, dfs.r)
    assert all(dfs.p0[v] == pred[v] for v in range(g.n) if v != dfs.r)


@pytest.mark.parametrize("name,n,want_f,want_steps", [("K2", 2, 1, 1), ("P3", 3, 6, 2)])
def test_tree_graphs_every_sample_is_exact(name, n, want_f, want_steps):
    """A graph that is itself a tree has one spanning tree: every sample is
    the graph, each non-root vertex departs once straight into the tree, and
    f = 2m K with K = sum_e vol_e (2m - vol_e) / 2m (Theorem 1 with one tree):
    K2 gives 1 * 1 / 2 = 1/2, so f = 1; P3 gives 2 * (1 * 3) / 4 = 3/2, f = 6."""
    g = S.complete(2) if name == "K2" else S.path(3)
    assert g.n == n and g.m == n - 1
    t0 = O.tau0(g)
    f, steps = O.sample_batch(g, t0, 5, 0, 32)
    assert f.tolist() == [want_f] * 32 and steps.tolist() == [want_steps] * 32
    assert want_f / (2 * g.m) == pytest.approx(O.K_dense(g), rel=1e-12)
