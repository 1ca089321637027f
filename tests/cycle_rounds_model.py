"""A CPU model of round-synchronous cycle popping (test infrastructure).

The alternative to walkers for parallelism inside one tree: every vertex
outside the tree holds its current arrow (its k-th draw); each round finds the
vertices whose arrows lead into the tree and redraws every vertex on a cycle of
the remaining arrows.  Each vertex's arrows form a stack and, by Wilson's
cycle-popping theorem, the set of popped cycles does not depend on the order in
which cycles are popped, so the final arrows are the tree of sequential Wilson
on the same stacks and the number of draws is its step count.  The model counts
rounds and the vertices still outside the tree summed over rounds: the work a
round-synchronous kernel would do.

    python tests/cycle_rounds_model.py 30 60 120     # perturbed grids, 3 trees each
"""
from __future__ import annotations

import math
import sys

import numpy as np


def pop_in_rounds(g, r: int, draw):
    """draw(vs, ks) gives the neighbour index (0 .. deg-1) of each vertex vs on
    its ks-th draw.  Returns (parent, draws, rounds, active vertex-rounds)."""
    n = g.n
    off = g.row_off
    k = np.zeros(n, dtype=np.int64)
    arrow = np.arange(n, dtype=np.int64)  # the root points at itself
    vs = np.flatnonzero(np.arange(n) != r)
    arrow[vs] = g.col[off[vs] + draw(vs, k[vs])]
    k[vs] = 1
    levels = max(1, math.ceil(math.log2(max(n, 2)))) + 1
    rounds = 0
    work = 0
    while True:
        # f^N with N >= n: the root for vertices whose arrows reach it, a
        # vertex of the cycle otherwise (f^N of the graph is its set of cycles)
        land = arrow.copy()
        for _ in range(levels):
            land = land[land]
        outside = np.flatnonzero(land != r)
        if outside.size == 0:
            break
        rounds += 1
        work += outside.size
        cyc = np.unique(land[outside])
        arrow[cyc] = g.col[off[cyc] + draw(cyc, k[cyc])]
        k[cyc] += 1
    parent = arrow.astype(np.int32)
    parent[r] = -1
    return parent, int(k.sum()), rounds, work


def philox_draw(g, seed: int, sample: int):
    """Draws of the walk stream: neighbour bounded(seed, v, k, sample, WALK, deg v)."""
    import oracle as O

    def draw(vs, ks):
        return np.array([O.bounded(seed, int(v), int(kk), sample, 0, int(g.deg[v]))
                         for v, kk in zip(vs, ks)], dtype=np.int64)
    return draw


def numpy_draw(g, seed: int):
    """Independent uniform draws from numpy (same distribution, faster)."""
    rng = np.random.default_rng(seed)

    def draw(vs, ks):
        return (rng.random(vs.shape[0]) * g.deg[vs]).astype(np.int64)
    return draw


def main(sides):
    import oracle as O
    from paper_2511_16356_gb300 import synth as S

    for side in sides:
        g = S.grid_perturbed(side, side, 0.25, 1)
        r = O.tau0(g).r
        rows = [pop_in_rounds(g, r, numpy_draw(g, s))[1:] for s in range(3)]
        print(f"{side}x{side} grid, 25% deleted: rounds {[x[1] for x in rows]}, "
              f"draws/n {[round(x[0] / g.n, 1) for x in rows]}, "
              f"active vertex-rounds/n {[round(x[2] / g.n, 1) for x in rows]}", flush=True)


if __name__ == "__main__":
    import os

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    main([int(a) for a in sys.argv[1:]] or [30, 60])
