"""Oracle: free-field (U = 1) Wilson propagator in closed form (test only).

For U = 1 a plane wave psi(x) = exp(i p.x) u is an eigenvector of the stencil
of oracle.wilson:  sum_mu [(1-g_mu) e^{i p_mu} + (1+g_mu) e^{-i p_mu}]
                  = sum_mu [2 cos p_mu - 2 i g_mu sin p_mu],
so D(p) = a(p) + i gamma.b(p),  a = 1 - 2 kappa sum_mu cos p_mu,
b_mu = 2 kappa sin p_mu, and D(p)^{-1} = (a - i gamma.b) / (a^2 + |b|^2).
Momenta: p_mu = 2 pi k / L_mu (periodic) or (2k+1) pi / L_mu (antiperiodic).
"""
import numpy as np

from .gamma import GAMMA, ID4


def momenta(L, bc):
    k = np.arange(L)
    return (2 * k + (1 if bc == -1 else 0)) * np.pi / L


def trace_inverse(dims, kappa, bc):
    """tr D^{-1} = 12 sum_p a / (a^2 + |b|^2)."""
    ps = [momenta(L, b) for L, b in zip(dims, bc)]
    P = np.meshgrid(*ps, indexing='ij')
    a = 1 - 2 * kappa * sum(np.cos(p) for p in P)
    b2 = sum((2 * kappa * np.sin(p)) ** 2 for p in P)
    return 12.0 * np.sum(a / (a * a + b2))


def point_propagator(dims, kappa, bc):
    """S(x) = D^{-1}(x, 0) as a 4x4 spin matrix (colour part is 1_3), shape
    (T, Z, Y, X, 4, 4): S(x) = (1/V) sum_p e^{i p.x} (a - i gamma.b)/(a^2 + |b|^2).
    The momentum sum is done one direction at a time with explicit phase
    matrices (a separable DFT)."""
    X, Y, Z, T = dims
    ps = [momenta(L, b) for L, b in zip(dims, bc)]
    P = np.meshgrid(*ps, indexing='ij')        # axes (px, py, pz, pt)
    a = 1 - 2 * kappa * sum(np.cos(p) for p in P)
    bs = [2 * kappa * np.sin(p) for p in P]
    den = a * a + sum(b * b for b in bs)
    M = np.einsum('...,st->...st', a / den, ID4)
    for mu in range(4):
        M = M - 1j * np.einsum('...,st->...st', bs[mu] / den, GAMMA[mu])
    # sum over p with phase e^{i p x}: apply per axis
    out = M
    for mu, L in enumerate(dims):
        x = np.arange(L)
        F = np.exp(1j * np.outer(x, ps[mu]))           # (x, p)
        out = np.moveaxis(np.tensordot(F, out, axes=([1], [mu])), 0, mu)
    out = out / (X * Y * Z * T)
    # axes now (x, y, z, t, s, s') -> (t, z, y, x, s, s')
    return np.ascontiguousarray(np.transpose(out, (3, 2, 1, 0, 4, 5)))


def pion_correlator(dims, kappa, bc):
    """C(t) = sum_{x in t} || D^{-1}(x; 0) ||_F^2 over the 12x12 spin-colour
    block (colour identity contributes a factor 3)."""
    S = point_propagator(dims, kappa, bc)
    return 3.0 * np.sum(np.abs(S) ** 2, axis=(1, 2, 3, 4, 5))
