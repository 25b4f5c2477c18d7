"""CPU-side checks of the C-ABI library: it loads, it exports every function
include/wd.h declares, argument validation needs no GPU, and the host-only
colouring search is bit-exact against the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, 'include', 'wd.h')).read()
    src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
    return sorted(set(re.findall(r'^\s*(?:int|int64_t|const char \*)\s*\**\s*(\w+)\s*\(', src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    from paper_2607_05157_b300 import _lib
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(_lib.lib, n), n
    assert set(names) == set(_lib.EXPORTED)


def test_bad_arguments_rejected_without_gpu():
    from paper_2607_05157_b300 import _lib
    h = ctypes.c_void_p()
    dims = (ctypes.c_int * 4)(4, 4, 3, 4)          # odd extent
    bc = (ctypes.c_int * 4)(1, 1, 1, -1)
    g = np.zeros(4 * 4 * 4 * 3 * 4 * 9, np.complex128)
    assert _lib.lib.wd_create(ctypes.byref(h), dims, g.ctypes.data, 0.1, bc, None) == _lib.WD_EINVAL
    assert b'even' in _lib.lib.wd_last_error()
    assert _lib.lib.wd_create(None, dims, g.ctypes.data, 0.1, bc, None) == _lib.WD_EINVAL


@pytest.mark.parametrize("dims,d", [((32, 32, 32), 1), ((32, 32, 32), 2), ((32, 32, 32), 3), ((32, 32, 32), 4),
                                    ((32, 32, 32, 64), 1), ((32, 32, 32, 64), 2), ((32, 32, 32, 64), 3),
                                    ((32, 32, 32, 64), 4), ((4, 4, 4, 4), 2), ((4, 4, 4, 4), 3),
                                    ((8, 8, 8, 16), 2), ((16, 16, 16, 32), 2), ((16, 16, 16, 32), 4),
                                    ((6, 4, 2, 8), 2), ((5, 7, 3), 2), ((12, 12, 12, 24), 2)])
def test_probe_color_bit_exact_vs_oracle(dims, d):
    from oracle import coloring
    from paper_2607_05157_b300 import probe_color
    nc, sigma, cols = probe_color(dims, d)
    onc, osig = coloring.search(dims, d, max_nc=4096)
    assert (nc, sigma) == (onc, osig)
    assert np.array_equal(cols, coloring.colors(dims, osig, onc))


def test_mlmc_allocate_matches_oracle():
    """Eq. 6 in libwd (host code, no GPU) against the oracle: identical
    integer sample counts, and bad arguments rejected."""
    import numpy as np
    from oracle import estimators
    from paper_2607_05157_b300 import mlmc_allocate, WDError
    assert list(mlmc_allocate([4.0, 1.0], [1.0, 4.0], 1.0)) == [8, 2]
    rng = np.random.default_rng(5)
    for _ in range(200):
        L = int(rng.integers(1, 6))
        V = rng.uniform(0.0, 50.0, L) * (rng.uniform(size=L) > 0.1)
        C = rng.uniform(0.01, 20.0, L)
        eps = float(rng.uniform(0.01, 2.0))
        _, ref = estimators.mlmc_allocation(V, C, eps)
        got = mlmc_allocate(V, C, eps)
        assert np.array_equal(got, ref), (V, C, eps, got, ref)
        assert np.sum(V / got) <= eps ** 2 * (1 + 1e-12)
    for V, C, eps in (([1.0], [0.0], 1.0), ([-1.0], [1.0], 1.0), ([1.0], [1.0], 0.0), ([1e30], [1e-30], 1e-20)):
        with pytest.raises(WDError):
            mlmc_allocate(V, C, eps)
