"""Pins of the oracle's sample maintenance (Sec. 4).

* BSM insertion theorem: E_{U(G')} f = (1 - R) E_{U(G)} f + R E_{U(G'_e)} f,
  and R = |Gamma'_e| / |Gamma'| (exhaustive enumeration on tiny graphs).
* Theorem 6 (link-cut) and Theorem 7 (cut-link) by enumerating the whole
  link-cut bipartite graph: every (tree, choice) pair through the oracle's own
  link_cut / cut_link; the reported degrees d(tau_e) / d(tau) must equal the
  in-degrees counted by enumeration, and the reweighted averages must satisfy the
  theorems to 1e-12.  Algorithm 3's deletion weight as printed (new/old) is
  biased; Theorem 7's (old/new) is not.
* Example 6's numbers (golden file).
* Whole updates: after BSM/ISM insertions and deletions (with refresh) the
  estimate over many trees is within a few standard errors of K(G').
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from oracle.dynamic import BSM, ISM, DynamicOracle
from paper_2511_16356_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _with_edge(g, u, v, add=True):
    e = {(int(a), int(b)) for a, b in g.edges()}
    key = (min(u, v), max(u, v))
    if add:
        e.add(key)
    else:
        e.remove(key)
    arr = np.array(sorted(e))
    return S.csr_from_edges(g.n, arr[:, 0], arr[:, 1])


def _fvals(g, t0, trees):
    out = {}
    for T in trees:
        p = O.orient(g.n, T, t0.r)
        out[tuple(sorted(T))] = O.f_alg1(g, t0, p, O.traverse(g, t0.r, p).vol)
    return out


def _key(p, r):
    return tuple(sorted((min(v, int(p[v])), max(v, int(p[v]))) for v in range(len(p)) if v != r))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bsm_insert_theorem(seed):
    g = S.random_connected(6, 0.5, seed)
    non = [(a, b) for a in range(g.n) for b in range(a + 1, g.n) if b not in set(g.neighbors(a))]
    u, v = non[0]
    g2 = _with_edge(g, u, v)
    t0 = O.tau0(g)  # tau0 of G stays a spanning tree of G'
    G1, G2 = O.spanning_trees(g), O.spanning_trees(g2)
    Ge = [T for T in G2 if (u, v) in T]
    R = O.resistance(g2, u, v)
    assert R == pytest.approx(len(Ge) / len(G2), rel=1e-12)
    f2 = _fvals(g2, t0, G2)
    lhs = np.mean([f2[tuple(sorted(T))] for T in G2])
    rhs = (1 - R) * np.mean([f2[tuple(sorted(T))] for T in G1]) + R * np.mean(
        [f2[tuple(sorted(T))] for T in Ge])
    assert lhs == pytest.approx(rhs, rel=1e-12)
    assert lhs / (2 * g2.m) == pytest.approx(O.K_dense(g2), rel=1e-12)


@pytest.mark.parametrize("seed", [4, 5, 6])
def test_theorem6_link_cut_enumeration(seed):
    g = S.random_connected(6, 0.55, seed)
    non = [(a, b) for a in range(g.n) for b in range(a + 1, g.n) if b not in set(g.neighbors(a))]
    u, v = non[-1]
    g2 = _with_edge(g, u, v)
    t0 = O.tau0(g)
    r = t0.r
    G1 = O.spanning_trees(g)
    Ge = [T for T in O.spanning_trees(g2) if (u, v) in T]
    R = O.resistance(g2, u, v)
    f2 = _fvals(g2, t0, Ge)
    indeg = {tuple(sorted(T)): 0 for T in Ge}
    dnew_of = {}
    acc = 0.0
    for T in G1:
        p = O.orient(g.n, T, r)
        _, d_old, _ = O.link_cut(g2, p, r, u, v, k_force=0)
        inner = 0.0
        for k in range(d_old):
            q, d_old2, d_new = O.link_cut(g2, p, r, u, v, k_force=k)
            assert d_old2 == d_old
            key = _key(q, r)
            assert key in indeg, "link-cut must give a spanning tree containing e"
            assert q[r] == -1
            indeg[key] += 1
            dnew_of.setdefault(key, d_new)
            assert dnew_of[key] == d_new
            inner += f2[key] * d_old / d_new
        acc += inner / d_old
    for key, c in indeg.items():
        assert c == dnew_of[key], "d(tau_e) must equal its in-degree in the link-cut graph"
    lhs = np.mean(list(f2.values()))
    rhs = (1 - R) / R * acc / len(G1)
    assert lhs == pytest.approx(rhs, rel=1e-12)


@pytest.mark.parametrize("seed", [7, 8, 9])
def test_theorem7_cut_link_enumeration(seed):
    g = S.random_connected(6, 0.6, seed)
    # an edge whose removal keeps g connected
    for a, b in g.edges():
        g2 = _with_edge(g, int(a), int(b), add=False)
        if S.is_connected(g2) and np.all(g2.deg > 0):
            u, v = int(a), int(b)
            break
    t0 = O.tau0(g2)
    r = t0.r
    Ge = [T for T in O.spanning_trees(g) if (u, v) in T]   # trees of G containing e
    G2 = O.spanning_trees(g2)
    R = O.resistance(g, u, v)
    f2 = _fvals(g2, t0, G2)
    indeg = {tuple(sorted(T)): 0 for T in G2}
    dnew_of = {}
    acc_thm7 = 0.0
    acc_printed = 0.0
    for T in Ge:
        p = O.orient(g.n, T, r)
        _, d_old, _ = O.cut_link(g2, p, r, u, v, k_force=0)
        i7 = ip = 0.0
        for k in range(d_old):
            q, d_old2, d_new = O.cut_link(g2, p, r, u, v, k_force=k)
            assert d_old2 == d_old
            key = _key(q, r)
            assert key in indeg and q[r] == -1
            indeg[key] += 1
            dnew_of.setdefault(key, d_new)
            assert dnew_of[key] == d_new
            i7 += f2[key] * d_old / d_new
            ip += f2[key] * d_new / d_old
        acc_thm7 += i7 / d_old
        acc_printed += ip / d_old
    for key, c in indeg.items():
        assert c == dnew_of[key], "d(tau) must equal its in-degree in the cut-link graph"
    lhs = np.mean(list(f2.values()))
    assert lhs == pytest.approx(R / (1 - R) * acc_thm7 / len(Ge), rel=1e-12)
    assert abs(lhs - R / (1 - R) * acc_printed / len(Ge)) > 1e-6 * abs(lhs)


def test_example6_weights():
    gold = {}
    for line in open(os.path.join(GOLDEN, "example6_linkcut.txt")):
        line = line.split("#")[0].split()
        if len(line) >= 3:
            gold[line[0]] = Fraction(int(line[1]), int(line[2]))
    out_deg = {1: 1, 2: 1, 3: 2}
    reach = {1: [4], 2: [4], 3: [4, 5]}
    in_deg = {4: 3, 5: 1}
    p = {4: Fraction(0), 5: Fraction(0)}
    e = {4: Fraction(0), 5: Fraction(0)}
    for t, nb in reach.items():
        assert len(nb) == out_deg[t]
        for te in nb:
            p[te] += Fraction(1, 3) * Fraction(1, out_deg[t])
            # link-cut weight d(tau)/d(tau_e), as in the oracle's ISM insertion
            e[te] += Fraction(1, 3) * Fraction(1, out_deg[t]) * Fraction(out_deg[t], in_deg[te])
    assert p[4] == gold["p_tau4"] and p[5] == gold["p_tau5"]
    assert e[4] == gold["E_tau4"] and e[5] == gold["E_tau5"]


def _sem(vals):
    return np.std(vals) / math.sqrt(len(vals))


@pytest.mark.parametrize("mode", [BSM, ISM])
def test_updates_keep_estimate_unbiased(mode):
    g = S.random_connected(9, 0.45, 12)
    non = [(a, b) for a in range(g.n) for b in range(a + 1, g.n) if b not in set(g.neighbors(a))]
    D = DynamicOracle(g, seed=31 + mode, n_trees=3000)
    u, v = non[1]
    D.insert(u, v, mode, refresh=True)
    k1 = O.K_dense(D.g)
    x = np.array(D.f, dtype=np.float64) / (2 * len(D.edges))
    w = np.array(D.w)
    est = D.estimate()
    # weighted standard error (effective sample size)
    neff = w.sum() ** 2 / (w ** 2).sum()
    se = math.sqrt(np.average((x - est) ** 2, weights=w) / neff)
    assert abs(est - k1) < 5 * se + 1e-9
    # then delete an edge that keeps the graph connected
    for a, b in D.g.edges():
        a, b = int(a), int(b)
        try:
            D.delete(a, b, mode, refresh=True)
            break
        except ValueError:
            continue
    k2 = O.K_dense(D.g)
    x = np.array(D.f, dtype=np.float64) / (2 * len(D.edges))
    w = np.array(D.w)
    est = D.estimate()
    neff = w.sum() ** 2 / (w ** 2).sum()
    se = math.sqrt(np.average((x - est) ** 2, weights=w) / neff)
    assert abs(est - k2) < 5 * se + 1e-9


def test_update_errors_and_tau0_rebuild():
    g = S.grid(4, 4)
    D = DynamicOracle(g, seed=3, n_trees=20)
    a, b = (0, 1)
    with pytest.raises(ValueError):
        D.insert(a, b, BSM)  # exists
    p = S.path(5)
    Dp = DynamicOracle(p, seed=1, n_trees=4)
    with pytest.raises(ValueError):
        Dp.delete(1, 2, BSM)  # bridge
    # deleting a tau0 edge rebuilds tau0 as the BFS tree of G'
    r = D.r
    child = int(next(v for v in range(g.n) if D.t0.p0[v] == r))
    D.delete(r, child, BSM)
    t0 = O.tau0(D.g, r)
    assert np.array_equal(D.t0.p0, t0.p0)
    assert all(not D.contains(k, r, child) for k in range(len(D.parents)))
