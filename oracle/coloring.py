"""Oracle: torus colouring (Sec. 3, Eq. 15; Table 1).  Test infrastructure only.

`search` wraps the exhaustive C search in coloring.c (compiled by `build`);
`colors` evaluates c(x) = sum_j sigma_j x_j mod n_c on a lattice;
`brute_force_valid` checks distance-d validity directly over all site pairs,
independently of the search's displacement enumeration.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, '_oracle_coloring.so')
_lib = None


def build(force=False):
    """Compile coloring.c with gcc into oracle/_oracle_coloring.so."""
    src = os.path.join(_HERE, 'coloring.c')
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        subprocess.check_call(['gcc', '-O2', '-shared', '-fPIC', '-o', _SO, src])
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
        for f in (_lib.oracle_torus_coloring, _lib.oracle_coloring_exists):
            f.restype = ctypes.c_int
            f.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                          ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    return _lib


def search(L, d, max_nc=4096):
    """(n_c, sigma) for torus extents L (n_D = len(L)) and distance d."""
    lib = _load()
    nD = len(L)
    Lc = (ctypes.c_int * nD)(*L)
    sig = (ctypes.c_int * nD)()
    nc = lib.oracle_torus_coloring(nD, Lc, d, max_nc, sig)
    return nc, tuple(sig[j] for j in range(nD))


def exists(L, d, nc):
    """Is there any sigma giving a valid distance-d colouring with exactly nc colours?"""
    lib = _load()
    nD = len(L)
    Lc = (ctypes.c_int * nD)(*L)
    sig = (ctypes.c_int * nD)()
    ok = lib.oracle_coloring_exists(nD, Lc, d, nc, sig)
    return bool(ok), tuple(sig[j] for j in range(nD))


def colors(L, sigma, nc):
    """c(x) for every site, as an int array over the lattice in lexicographic
    order (first coordinate fastest): index = x_0 + L_0 (x_1 + L_1 (...))."""
    grids = np.meshgrid(*[np.arange(l) for l in L], indexing='ij')
    c = sum(s * g for s, g in zip(sigma, grids)) % nc
    # meshgrid 'ij' puts x_0 slowest; transpose so x_0 is fastest in C order
    return np.ascontiguousarray(np.transpose(c)).reshape(-1).astype(np.int32)


def brute_force_valid(L, col, d):
    """True iff no two distinct sites within torus L1 distance d share a colour.
    col is indexed lexicographically with the first coordinate fastest."""
    L = list(L)
    V = int(np.prod(L))
    idx = np.arange(V)
    coords = []
    rem = idx.copy()
    for l in L:
        coords.append(rem % l); rem //= l
    coords = np.array(coords)           # (nD, V)
    for s in range(V):
        diff = np.abs(coords - coords[:, s:s + 1])
        tdist = np.minimum(diff, np.array(L)[:, None] - diff).sum(axis=0)
        close = (tdist <= d) & (idx != s)
        if np.any(col[close] == col[s]):
            return False
    return True
