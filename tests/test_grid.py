"""Activity-quantile grids: the library's host split against the oracle's
independent one, and a hand-worked example."""
import numpy as np
import pytest

import oracle
from paper_1907_07410_gb300 import grid


def test_hand_example():
    # counts per id: [5, 1, 3, 0, 3] -> order 0, 2, 4, 1, 3 (ties by id)
    ids = np.array([0] * 5 + [1] + [2] * 3 + [4] * 3)
    perm, bounds = grid.quantile_split(ids, 5, 2)
    assert perm.tolist() == [0, 3, 1, 4, 2]
    # ratings before positions 0..5: 0, 5, 8, 11, 12, 12; half of 12 is
    # first reached before position 2
    assert bounds.tolist() == [0, 2, 5]
    perm3, bounds3 = grid.quantile_split(ids, 5, 3)
    # thirds: 4 and 8 ratings -> positions 1 (5 >= 4) and 2 (8 >= 8)
    assert bounds3.tolist() == [0, 1, 2, 5]


@pytest.mark.parametrize("seed,size,parts", [(1, 50, 4), (2, 1000, 8),
                                             (3, 300, 32), (4, 17, 17)])
def test_matches_oracle(seed, size, parts):
    rng = np.random.default_rng(seed)
    w = (np.arange(size) + 1.0) ** -1.1
    ids = rng.choice(size, size=20 * size, p=w / w.sum())
    perm, bounds = grid.quantile_split(ids, size, parts)
    operm, obounds = oracle.activity_quantile_cut(ids, size, parts)
    assert np.array_equal(perm, operm)
    assert np.array_equal(bounds, obounds)
    assert bounds[0] == 0 and bounds[-1] == size
    assert np.all(np.diff(bounds) >= 0)
    assert np.array_equal(np.sort(perm), np.arange(size))


def test_oracle_cut_hand_example():
    ids = np.array([0] * 5 + [1] + [2] * 3 + [4] * 3)
    perm, bounds = oracle.activity_quantile_cut(ids, 5, 2)
    assert perm.tolist() == [0, 3, 1, 4, 2]
    assert bounds.tolist() == [0, 2, 5]
    assert oracle.activity_quantile_cut(ids, 5, 3)[1].tolist() == [0, 1, 2, 5]


@pytest.mark.parametrize("seed,size,parts", [(5, 40, 3), (6, 200, 7)])
def test_oracle_cut_brute_force(seed, size, parts):
    """Each bound is the first position whose preceding ids hold at least
    g / parts of the ratings, checked by trying every position; the order is
    by count descending, ids ascending on ties."""
    rng = np.random.default_rng(seed)
    ids = rng.integers(0, size, size=15 * size) ** 2 % size
    perm, bounds = oracle.activity_quantile_cut(ids, size, parts)
    counts = np.bincount(ids, minlength=size)
    order = np.argsort(perm)
    for a, b in zip(order[:-1], order[1:]):
        assert (counts[a], -a) > (counts[b], -b)
    total = len(ids)
    for g in range(1, parts):
        first = next(j for j in range(size + 1)
                     if parts * counts[order[:j]].sum() >= g * total)
        assert bounds[g] == first
