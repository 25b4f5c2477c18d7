"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *draws* arrays: SU(3) gauge fields shaped like the lattices of
the paper's workloads, and Gaussian test spinors.  It holds none of the trace
estimators' arithmetic (no stencil, no noise hash, no colouring): those are
written separately by the oracle and by the CUDA path.

Array conventions (the C boundary uses the same ones):
  * lattice dims are given as (X, Y, Z, T); site index = x + X*(y + Y*(z + Z*t));
  * a gauge field is complex128 of shape (4, T, Z, Y, X, 3, 3), entry
    [mu, t, z, y, x, a, b] = U_mu(x)_{ab}  (row = colour a), mu = 0..3 <-> x,y,z,t;
  * a spinor batch is complex128 of shape (nrhs, T, Z, Y, X, 4, 3)
    (spin index before colour index).

The paper's ensemble (RQCD ensemble IV, a 64x32^3 gauge configuration) is not
available, so every field here is a synthetic stand-in: each link is the SU(3)
projection of I + s*G with G a complex Gaussian 3x3 matrix (s = "spread").
"""
import numpy as np


def gauge_field(dims, spread, seed):
    """Random SU(3) links: Gram-Schmidt on the columns of I + spread*G, then
    divide by the principal cube root of the determinant (det U = 1).

    G has independent N(0,1) real and imaginary parts drawn from
    numpy.random.default_rng(seed) in the order (mu, t, z, y, x, a, b, re/im).
    spread = 0 gives the free field U = 1.
    """
    X, Y, Z, T = dims
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((4, T, Z, Y, X, 3, 3, 2))
    m = np.eye(3) + spread * (g[..., 0] + 1j * g[..., 1])
    u = np.empty_like(m)
    # classical Gram-Schmidt on columns 0, 1, 2
    c0 = m[..., :, 0]
    c0 = c0 / np.linalg.norm(c0, axis=-1, keepdims=True)
    c1 = m[..., :, 1]
    c1 = c1 - np.sum(c0.conj() * c1, axis=-1, keepdims=True) * c0
    c1 = c1 / np.linalg.norm(c1, axis=-1, keepdims=True)
    c2 = m[..., :, 2]
    c2 = (c2 - np.sum(c0.conj() * c2, axis=-1, keepdims=True) * c0
             - np.sum(c1.conj() * c2, axis=-1, keepdims=True) * c1)
    c2 = c2 / np.linalg.norm(c2, axis=-1, keepdims=True)
    u[..., :, 0], u[..., :, 1], u[..., :, 2] = c0, c1, c2
    det = np.linalg.det(u)
    u = u / (det ** (1.0 / 3.0))[..., None, None]   # principal cube root
    return np.ascontiguousarray(u)


def unit_gauge(dims):
    """The free field U_mu(x) = 1."""
    X, Y, Z, T = dims
    u = np.zeros((4, T, Z, Y, X, 3, 3), np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def spinors(dims, nrhs, seed):
    """Complex Gaussian spinors, shape (nrhs, T, Z, Y, X, 4, 3)."""
    X, Y, Z, T = dims
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((nrhs, T, Z, Y, X, 4, 3, 2))
    return np.ascontiguousarray(g[..., 0] + 1j * g[..., 1])


def su3_algebra(dims, seed):
    """Random traceless Hermitian 3x3 matrices on every link, each normalised
    to unit Frobenius norm; shape (4, T, Z, Y, X, 3, 3).  Used as the link
    directions of finite-difference gradient checks (U -> exp(i h T) U)."""
    X, Y, Z, T = dims
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((4, T, Z, Y, X, 3, 3, 2))
    a = g[..., 0] + 1j * g[..., 1]
    h = 0.5 * (a + np.swapaxes(a.conj(), -1, -2))
    tr = np.trace(h, axis1=-2, axis2=-1)
    h = h - tr[..., None, None] * np.eye(3) / 3.0
    return h / np.linalg.norm(h, axis=(-2, -1), keepdims=True)


def test_vectors(dims, nv, seed):
    """nv complex Gaussian fine-lattice vectors, shape (nv, T, Z, Y, X, 4, 3).
    Random starting vectors for the multigrid setup."""
    return spinors(dims, nv, seed)
