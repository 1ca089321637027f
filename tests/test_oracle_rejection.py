"""Pins of sampling with rejection by walk length (oracle.accepted_samples).

The claim: the tree Wilson's algorithm returns is independent of its step
count S, so trees accepted by any rule on S are still uniform and f/2m stays
unbiased for K.

* Exact: every run of sequential Wilson with at most s_max departures is
  enumerated with its rational probability on small graphs; for every s the
  probability P(T, S = s) is the same for all spanning trees T, and the mean of
  f over the trees with S <= X equals 2m K.
* Statistical: on the 3x3 grid (192 trees) the oracle's trees with S at most
  the median and those above it each pass a chi-square test of uniformity.
* The sampler's bookkeeping: accepted ids ascend, every accepted tree has
  S <= cap, every skipped id has S > cap.
"""
from collections import defaultdict
from fractions import Fraction

import numpy as np
import pytest
from scipy.stats import chi2

import oracle as O
from paper_2511_16356_gb300 import synth as S


def _joint_tree_steps(g, r, s_max):
    """{(tree edges, S): probability} over runs of Wilson (starts in id order)
    with S <= s_max; exact fractions."""
    n = g.n
    nbrs = [[int(w) for w in g.col[g.row_off[v]:g.row_off[v + 1]]] for v in range(n)]
    out = defaultdict(Fraction)

    def start(intree, parent, idx, steps, prob):
        while idx < n and intree[idx]:
            idx += 1
        if idx == n:
            key = tuple(sorted((min(v, parent[v]), max(v, parent[v])) for v in range(n) if v != r))
            out[(key, steps)] += prob
            return
        walk(intree, parent, idx, [idx], steps, prob)

    def walk(intree, parent, idx, path, steps, prob):
        if steps >= s_max:
            return
        u = path[-1]
        p = prob / len(nbrs[u])
        for w in nbrs[u]:
            if intree[w]:
                it2, par2 = list(intree), list(parent)
                for i, x in enumerate(path):
                    par2[x] = path[i + 1] if i + 1 < len(path) else w
                    it2[x] = True
                start(it2, par2, idx + 1, steps + 1, p)
            elif w in path:
                walk(intree, parent, idx, path[:path.index(w) + 1], steps + 1, p)
            else:
                walk(intree, parent, idx, path + [w], steps + 1, p)

    intree = [v == r for v in range(n)]
    start(intree, [-1] * n, 0, 0, Fraction(1))
    return out


@pytest.mark.parametrize("name,s_max", [("K4", 9), ("C5", 12), ("grid2x3", 10), ("K2,3", 10)])
def test_tree_is_independent_of_step_count_exactly(name, s_max):
    g = {"K4": lambda: S.complete(4), "C5": lambda: S.cycle(5), "grid2x3": lambda: S.grid(2, 3),
         "K2,3": lambda: S.complete_bipartite(2, 3)}[name]()
    t0 = O.tau0(g)
    trees = [tuple(sorted(T)) for T in O.spanning_trees(g)]
    joint = _joint_tree_steps(g, t0.r, s_max)
    by_s = defaultdict(dict)
    for (T, s), p in joint.items():
        by_s[s][T] = p
    seen = 0
    for s, row in by_s.items():
        assert set(row) == set(trees), s          # every tree occurs at every step count seen
        assert len(set(row.values())) == 1, s     # with the same probability
        seen += 1
    assert seen >= 3
    assert sum(joint.values()) <= 1
    # the mean of f over trees accepted by S <= X is 2m K, for every X
    fs = {}
    for T in trees:
        par = O.orient(g.n, T, t0.r)
        fs[T] = O.f_alg1(g, t0, par, O.traverse(g, t0.r, par).vol)
    k_exact = O.K_dense(g)
    for X in sorted(by_s)[1:]:
        acc = defaultdict(Fraction)
        for (T, s), p in joint.items():
            if s <= X:
                acc[T] += p
        mean_f = sum(fs[T] * p for T, p in acc.items()) / sum(acc.values())
        assert float(mean_f) / (2 * g.m) == pytest.approx(k_exact, rel=1e-12)


def test_accepted_trees_are_uniform_chi_square():
    g = S.grid(3, 3)
    t0 = O.tau0(g)
    trees = O.spanning_trees(g)
    idx = {tuple(sorted(T)): i for i, T in enumerate(trees)}
    N = 400 * len(trees)
    steps = np.zeros(N, dtype=np.int64)
    which = np.zeros(N, dtype=np.int64)
    for k in range(N):
        par, st = O.wilson(g, t0.r, 4242, k)
        steps[k] = st
        which[k] = idx[tuple(sorted((min(v, int(par[v])), max(v, int(par[v])))
                                    for v in range(g.n) if v != t0.r))]
    med = np.median(steps)
    for part in (steps <= med, steps > med):
        cnt = np.bincount(which[part], minlength=len(trees)).astype(np.float64)
        e = part.sum() / len(trees)
        stat = ((cnt - e) ** 2 / e).sum()
        assert chi2.sf(stat, len(trees) - 1) > 1e-3


def test_accepted_samples_bookkeeping():
    g = S.grid_perturbed(8, 7, 0.2, 3)
    t0 = O.tau0(g)

    def sample(first, k):
        return O.sample_batch(g, t0, 9, first, k)

    f_all, s_all = sample(0, 600)
    cap = int(np.median(s_all))
    ids, f, steps = O.accepted_samples(sample, cap, 200, block=64)
    assert len(ids) == 200 and np.all(np.diff(ids) > 0) and np.all(steps <= cap)
    assert np.array_equal(f, f_all[ids]) and np.array_equal(steps, s_all[ids])
    skipped = np.setdiff1d(np.arange(ids[-1] + 1), ids)
    assert np.all(s_all[skipped] > cap)
