"""CPU check of the round-synchronous cycle-popping model
(tests/cycle_rounds_model.py): on the walk stream it ends with sequential
Wilson's tree and step count, for trees of several graph shapes."""
import numpy as np
import pytest

import oracle as O
from paper_2511_16356_gb300 import synth as S

from cycle_rounds_model import philox_draw, pop_in_rounds


@pytest.mark.parametrize("make", [lambda: S.grid_perturbed(9, 8, 0.25, 2), lambda: S.complete(9),
                                  lambda: S.er_lcc(80, 0.05, 3), lambda: S.cycle(25),
                                  lambda: S.star(7)])
def test_rounds_reproduce_sequential_wilson(make):
    g = make()
    t0 = O.tau0(g)
    for sample in range(3):
        parent, draws, rounds, work = pop_in_rounds(g, t0.r, philox_draw(g, 21, sample))
        ref = O.tree(g, t0, 21, sample)
        assert np.array_equal(parent, ref.parent)
        assert draws == ref.steps
        assert (rounds == 0) == (work == 0)
