"""Pins of the torus colouring (Sec. 3, Eq. 15) against Table 1 and brute force."""
import os

import numpy as np
import pytest

from oracle import coloring

GOLD = os.path.join(os.path.dirname(__file__), 'golden', 'table1_colors.txt')


def _table1():
    return [tuple(int(v) for v in l.split()) for l in open(GOLD) if l.strip() and not l.startswith('#')]


@pytest.mark.parametrize("nD,d,paper,reading", _table1())
def test_table1(nD, d, paper, reading):
    dims = (32, 32, 32) if nD == 3 else (32, 32, 32, 64)
    nc, sigma = coloring.search(dims, d)
    assert nc == reading
    if paper != reading:
        # the printed count admits no torus-valid sigma at all
        assert not coloring.exists(dims, d, paper)[0]


@pytest.mark.parametrize("dims,d", [((4, 4, 4, 4), 1), ((4, 4, 4, 4), 2), ((4, 4, 4, 4), 3),
                                    ((6, 4, 2, 8), 2), ((8, 8, 8), 3), ((5, 7, 3), 2),
                                    ((8, 8, 8, 16), 2)])
def test_search_result_is_valid_by_brute_force(dims, d):
    nc, sigma = coloring.search(dims, d, max_nc=512)
    col = coloring.colors(dims, sigma, nc)
    assert coloring.brute_force_valid(dims, col, d)
    # minimality: every smaller count fails for every sigma
    assert nc == 2 or not coloring.exists(dims, d, nc - 1)[0]


def test_brute_force_rejects_invalid():
    dims = (4, 4, 4, 4)
    col = coloring.colors(dims, (1, 1, 1, 1), 2)         # valid for d = 1 only
    assert coloring.brute_force_valid(dims, col, 1)
    assert not coloring.brute_force_valid(dims, col, 2)


def test_lexicographic_order_on_small_torus():
    """The search returns the lexicographically first valid sigma: check by a
    flat scan of all sigma in Python on a tiny torus."""
    import itertools
    dims, d = (4, 6, 2), 2
    nc, sigma = coloring.search(dims, d)
    for s in itertools.product(range(nc), repeat=3):
        if coloring.brute_force_valid(dims, coloring.colors(dims, s, nc), d):
            assert tuple(s) == sigma
            break
