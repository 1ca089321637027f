"""The wave makespan planning model (tests/wave_makespan_model.py): list
scheduling on identical slots, and the accounting of rejected trees."""
import pytest

from wave_makespan_model import makespan, wave_with_cap


def test_equal_jobs_fill_slots_in_rounds():
    assert makespan([2.0] * 10, 4) == 6.0   # rounds of 4, 4, 2 jobs
    assert makespan([5.0, 1.0, 1.0, 1.0], 2) == 5.0
    assert makespan([], 3) == 0.0


def test_rejected_trees_cost_the_cap_and_do_not_count():
    s = [1, 9, 1, 9, 1]
    # cap 4: trees 0, 2, 4 accepted; trees 1 and 3 stop at 4
    assert wave_with_cap(s, 3, 1, 1.0, cap=4) == 1 + 4 + 1 + 4 + 1
    assert wave_with_cap(s, 3, 1, 1.0) == 1 + 9 + 1
    with pytest.raises(ValueError):
        wave_with_cap(s, 4, 1, 1.0, cap=4)
