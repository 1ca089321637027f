"""CPU check of the parked-path walker design (tests/walker_park_model.py):
with P path slots served by L lanes, lanes parking confirmed waits and taking
other work, the protocol still pops exactly the cycles of sequential Wilson,
so tree, step count, depths and a parent-first order are the oracle's."""
import numpy as np
import pytest

import oracle as O
from paper_2511_16356_gb300 import synth as S

from walker_park_model import walk_tree_parked

GRAPHS = {
    "grid12x10p": lambda: S.grid_perturbed(12, 10, 0.25, 2),
    "er120": lambda: S.er_lcc(120, 0.04, 1),
    "K12": lambda: S.complete(12),
    "C30": lambda: S.cycle(30),
    "cl500": lambda: S.chung_lu(500, 2.1, 6.0, 4),
}


@pytest.mark.parametrize("lanes,slots", [(32, 32), (32, 64), (3, 8), (8, 128)])
@pytest.mark.parametrize("name", list(GRAPHS))
def test_parked_paths_reproduce_sequential_wilson(name, lanes, slots):
    g = GRAPHS[name]()
    t0 = O.tau0(g)
    rng = np.random.default_rng(9)
    for sample, sorder in enumerate([rng.permutation(g.n),
                                     np.lexsort((rng.permutation(g.n), t0.level))]):
        parent, steps, depth, order, _ = walk_tree_parked(g, t0.r, 31, sample, sorder,
                                                          lanes, slots)
        ref = O.tree(g, t0, 31, sample)
        assert np.array_equal(parent, ref.parent)
        assert steps == ref.steps
        assert np.array_equal(depth, ref.depth)
        where = np.empty(g.n, dtype=np.int64)
        where[order] = np.arange(g.n)
        assert all(where[parent[v]] < where[v] for v in range(g.n) if v != t0.r)
