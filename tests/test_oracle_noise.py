"""Pins of the oracle's Rademacher generator (Sec. 1, Eq. 1)."""
import os

import numpy as np

from oracle import noise

GOLD = os.path.join(os.path.dirname(__file__), 'golden', 'splitmix64.txt')
GOLDEN_RATIO = 0x9E3779B97F4A7C15


def test_splitmix64_published_values():
    lines = [l.split() for l in open(GOLD) if l.strip() and not l.startswith('#')]
    for row in lines:
        seed = int(row[0])
        outs = [int(v, 0) for v in row[1:]]
        keys = np.array([(seed + k * GOLDEN_RATIO) % 2 ** 64 for k in range(len(outs))], np.uint64)
        with np.errstate(over='ignore'):
            got = noise.splitmix64(keys)
        assert [int(g) for g in got] == outs


def test_rademacher_moments():
    """E[eta_j] = 0 and E[eta_j eta_k] = delta_jk (Eq. 1), checked statistically
    over 2000 samples of length 64: means within 5 sigma of 0."""
    n, N = 64, 2000
    E = np.array([noise.rademacher(17, i, n) for i in range(N)])
    assert set(np.unique(E)) == {-1.0, 1.0}
    assert np.abs(E.mean(axis=0)).max() < 5 / np.sqrt(N)
    C = E.T @ E / N
    off = C - np.diag(np.diag(C))
    assert np.allclose(np.diag(C), 1.0)
    assert np.abs(off).max() < 5 / np.sqrt(N)


def test_streams_differ():
    a = noise.rademacher(5, 0, 4096)
    b = noise.rademacher(5, 1, 4096)
    c = noise.rademacher(5, noise.COARSE_STREAM, 4096)
    assert 0.4 < np.mean(a != b) < 0.6 and 0.4 < np.mean(a != c) < 0.6
