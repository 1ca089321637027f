"""Pins of the oracle's two random choices of sample maintenance (Sec. 4).

* Algorithm 2 (and 3) replace / transform "randomly selected" ceil(R |S|) trees
  of the pool: `oracle.select` (Floyd's sampling on the select stream) must be
  a uniform k-subset of the N pool indices.  For every N <= 7 and every k the
  subsets drawn over many update sequence numbers are compared with the
  uniform law on all C(N, k) subsets by a chi-square test; every draw must be
  k distinct indices in [0, N).
* Algorithm 2's insertion draws Wilson(G', (u, v)), a uniform spanning tree of
  G' conditioned on containing the inserted edge, re-rooted at r: every output
  of `oracle.cond_wilson` must be a spanning tree rooted at r that contains
  (u, v), and its frequencies over the enumerated trees containing (u, v)
  must pass a chi-square test of uniformity.

A wrong bound or collision rule in the selection, or a conditioned walk that
starts from the wrong pre-rooted pair or skips the re-rooting, fails here.
"""
import itertools
import math

import numpy as np
import pytest
from scipy.stats import chi2

import oracle as O
from paper_2511_16356_gb300 import synth as S

P_MIN = 1e-3


@pytest.mark.parametrize("N", range(1, 8))
def test_select_is_a_uniform_k_subset(N):
    seed = 0x5E1EC7 + N
    for k in range(0, N + 1):
        subsets = list(itertools.combinations(range(N), k))
        idx = {s: i for i, s in enumerate(subsets)}
        draws = 200 * len(subsets) if len(subsets) > 1 else 50
        cnt = np.zeros(len(subsets))
        for seq in range(draws):
            out = [int(x) for x in O.select(seed, seq, N, k)]
            assert len(out) == k
            assert len(set(out)) == k, (N, k, seq, out)
            assert all(0 <= x < N for x in out), (N, k, seq, out)
            cnt[idx[tuple(sorted(out))]] += 1
        if len(subsets) == 1:
            continue  # k = 0 or k = N: the only subset, checked above
        e = draws / len(subsets)
        stat = ((cnt - e) ** 2 / e).sum()
        assert chi2.sf(stat, len(subsets) - 1) > P_MIN, (N, k, cnt)


def test_select_each_index_equally_often_on_a_larger_pool():
    """Marginals: P(i selected) = k / N for every i (N = 50, k = 13)."""
    N, k, draws = 50, 13, 20000
    hits = np.zeros(N)
    for seq in range(draws):
        hits[O.select(99, seq, N, k)] += 1
    p = k / N
    sd = math.sqrt(draws * p * (1 - p))
    assert np.all(np.abs(hits - draws * p) < 5 * sd), hits


def _tree_key(parent, r):
    return tuple(sorted((min(v, int(parent[v])), max(v, int(parent[v])))
                        for v in range(parent.shape[0]) if v != r))


def _rooted_spanning_tree(parent, r):
    n = parent.shape[0]
    if parent[r] != -1:
        return False
    for v in range(n):
        x, hops = v, 0
        while x != r:
            x = int(parent[x])
            hops += 1
            if x < 0 or hops > n:
                return False
    return True


@pytest.mark.parametrize("name,e,r_kind", [
    ("K4", (0, 1), "root"), ("K4", (2, 3), "root"),
    ("grid3x3", (4, 5), "root"), ("grid3x3", (0, 1), "far"),
    ("rc7", None, "root"), ("rc7", None, "far"),
])
def test_cond_wilson_uniform_over_trees_containing_e(name, e, r_kind):
    g = {"K4": S.complete(4), "grid3x3": S.grid(3, 3),
         "rc7": S.random_connected(7, 0.5, 3)}[name]
    edges = [tuple(map(int, x)) for x in g.edges()]
    if e is None:
        e = edges[len(edges) // 2]
    u, v = e
    assert (min(u, v), max(u, v)) in edges
    r = O.tau0(g).r if r_kind == "root" else max(x for x in range(g.n) if x not in (u, v))
    trees = [tuple(sorted(T)) for T in O.spanning_trees(g)]
    with_e = [T for T in trees if (min(u, v), max(u, v)) in T]
    assert 0 < len(with_e) < len(trees)
    idx = {T: i for i, T in enumerate(with_e)}
    N = 200 * len(with_e)
    cnt = np.zeros(len(with_e))
    seed = 4242 + len(name) + u * 7 + v
    for k in range(N):
        par, steps = O.cond_wilson(g, u, v, r, seed, k)
        assert _rooted_spanning_tree(par, r), (k, par)
        key = _tree_key(par, r)
        assert key in idx, (k, key)  # a spanning tree of g that contains (u, v)
        assert steps >= g.n - 2  # every vertex but u and v departs at least once
        cnt[idx[key]] += 1
    ex = N / len(with_e)
    stat = ((cnt - ex) ** 2 / ex).sum()
    assert chi2.sf(stat, len(with_e) - 1) > P_MIN, cnt


def test_cond_wilson_on_a_path_graph_is_forced():
    """On a tree graph there is one spanning tree: every conditioned draw returns
    it, oriented towards r."""
    g = S.path(6) if hasattr(S, "path") else None
    if g is None:
        pytest.skip("no path generator")
    for r in (0, 3, 5):
        want = O.orient(g.n, [tuple(map(int, x)) for x in g.edges()], r)
        for k in range(20):
            par, _ = O.cond_wilson(g, 2, 3, r, 7, k)
            assert np.array_equal(par, want)
