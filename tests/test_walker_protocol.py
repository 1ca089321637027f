"""CPU check of the 32-walker protocol's design (tests/walker_protocol_model.py):
for any start order and any number of walkers the concurrent protocol pops
exactly the cycles of sequential Wilson, so the tree, the step count, the
depths and a parent-first order come out as the oracle's (128 walkers: the
walker count of a four-warp, CTA-level version of the protocol)."""
import numpy as np
import pytest

import oracle as O
from paper_2511_16356_gb300 import synth as S

from walker_protocol_model import walk_tree

GRAPHS = {
    "er120": lambda: S.er_lcc(120, 0.04, 1),
    "grid9x7": lambda: S.grid(9, 7),
    "K12": lambda: S.complete(12),
    "C30": lambda: S.cycle(30),
    "star20": lambda: S.star(20),
    "grid15x11p": lambda: S.grid_perturbed(15, 11, 0.25, 2),
    "cl600": lambda: S.chung_lu(600, 2.1, 6.0, 4),
}


@pytest.mark.parametrize("lanes", [32, 3, 128])
@pytest.mark.parametrize("order_kind", ["random", "level", "ascending"])
@pytest.mark.parametrize("name", list(GRAPHS))
def test_concurrent_walkers_reproduce_sequential_wilson(name, order_kind, lanes):
    g = GRAPHS[name]()
    t0 = O.tau0(g)
    rng = np.random.default_rng(5)
    if order_kind == "random":
        sorder = rng.permutation(g.n)
    elif order_kind == "level":  # walkers start next to each other: many waits
        sorder = np.lexsort((rng.permutation(g.n), t0.level))
    else:
        sorder = np.arange(g.n)
    for sample in range(2):
        parent, steps, depth, order, _ = walk_tree(g, t0.r, 77, sample, sorder, lanes=lanes)
        ref = O.tree(g, t0, 77, sample)
        assert np.array_equal(parent, ref.parent)
        assert steps == ref.steps
        assert np.array_equal(depth, ref.depth)
        where = np.empty(g.n, dtype=np.int64)
        where[order] = np.arange(g.n)
        assert all(where[parent[v]] < where[v] for v in range(g.n) if v != t0.r)
