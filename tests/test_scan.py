"""Host logic of penalty scans: optimal and critical penalties from a
success table (no GPU)."""
import math

import numpy as np

from paper_1603_03755_gb300.scan import critical_penalty, optimal_penalty


def test_optimal_penalty_takes_the_smallest_of_ties_and_any_order():
    pens = [8, 2, 4, 6]
    succ = np.array([[0.3, 0.9], [0.1, 0.9], [0.5, 0.2], [0.5, 0.9]])   # rows follow pens
    assert list(optimal_penalty(pens, succ)) == [4.0, 2.0]


def test_critical_penalty_interpolates_the_first_crossing():
    pens = [1, 2, 4, 8]
    succ = np.array([[0.0, 0.6, 0.1, 0.0],
                     [0.2, 0.7, 0.3, 0.1],
                     [0.8, 0.9, 0.6, 0.2],
                     [0.4, 1.0, 0.9, 0.3]])
    got = critical_penalty(pens, succ)
    assert math.isclose(got[0], 2 + (0.5 - 0.2) * (4 - 2) / (0.8 - 0.2))    # first crossing, not the dip after
    assert got[1] == 1.0                                                     # starts above the level
    assert math.isclose(got[2], 2 + (0.5 - 0.3) * 2 / (0.6 - 0.3))
    assert math.isnan(got[3])                                                # never reaches 0.5
    # unsorted input gives the same answer
    perm = [2, 0, 3, 1]
    assert np.allclose(critical_penalty(np.array(pens)[perm], succ[perm]), got, equal_nan=True)
