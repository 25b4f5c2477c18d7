"""Oracle: derivatives of the trace estimates (test infrastructure only).

The paper has no gradients; they follow from differentiating its quadratic
forms.  For X = v^dag B D^{-1} v with z = D^{-1} v and w = D^{-dag} B^dag v,
    dX = - w^dag (dD) z.
With the stencil of oracle.wilson, a link change U_mu(x) -> U_mu(x) + h Delta_mu(x)
changes D by -kappa [(1-g_mu) Delta psi(x+mu) + (1+g_mu) Delta^dag psi(x-mu)]
on the two hops that use the link, hence
    dX/dh = sum_{x,mu} tr(Delta_mu(x) G_mu(x)) + conj(tr(Delta_mu(x) H_mu(x)))
with the per-link force matrices (3x3 colour outer products, spin summed)
    G_mu(x) = kappa b sum_s z(x+mu)_s  [(1-g_mu) w(x)]_s^dag
    H_mu(x) = kappa b sum_s [(1+g_mu) w(x+mu)]_s  z(x)_s^dag
where b = bc[mu] on the links that wrap around the lattice and 1 elsewhere.
For kappa: dD/dkappa = -H = (D - 1)/kappa, so dX/dkappa = (w^dag z - X)/kappa.
"""
import numpy as np

from .gamma import GAMMA, ID4
from .wilson import _AX, _shift, sparse_matrix


def link_force(w, z, kappa, bc):
    """(G, H), each (4, T, Z, Y, X, 3, 3); w, z: (..., T, Z, Y, X, 4, 3), a
    leading batch axis (several RHS) is summed over."""
    w = w.reshape((-1,) + w.shape[-6:])
    z = z.reshape((-1,) + z.shape[-6:])
    T, Z, Y, X = w.shape[1:5]
    G = np.zeros((4, T, Z, Y, X, 3, 3), np.complex128)
    H = np.zeros_like(G)
    for mu in range(4):
        zf = _shift(z, mu, +1, bc)          # bc[mu] * z(x+mu) on wrapped sites
        wf = _shift(w, mu, +1, (1, 1, 1, 1))
        pw = np.einsum('st,...tc->...sc', ID4 - GAMMA[mu], w)
        qw = np.einsum('st,...tc->...sc', ID4 + GAMMA[mu], wf)
        G[mu] = kappa * np.einsum('n...sa,n...sb->...ab', zf, pw.conj())
        # H needs the wrap factor once: apply it to z(x)'s partner w(x+mu) sites
        Hm = kappa * np.einsum('n...sa,n...sb->...ab', qw, z.conj())
        if bc[mu] != 1:
            idx = [slice(None)] * Hm.ndim
            idx[_AX[mu]] = Hm.shape[_AX[mu]] - 1
            Hm[tuple(idx)] *= bc[mu]
        H[mu] = Hm
    return G, H


def directional(G, H, Delta):
    """sum_{x,mu} tr(Delta G) + conj(tr(Delta H)) for link directions Delta."""
    a = np.einsum('...ab,...ba->...', Delta, G).sum()
    b = np.einsum('...ab,...ba->...', Delta, H).sum()
    return a + np.conj(b)


def hopping_derivative(Delta, kappa, bc):
    """dD/dh for U -> U + h Delta, as a sparse matrix (D is affine in the links)."""
    import scipy.sparse as sp
    n = 12 * int(np.prod(Delta.shape[1:5]))
    return sparse_matrix(Delta, kappa, bc) - sp.identity(n, dtype=np.complex128, format='csr')


def exact_derivative(Dinv, Bdiag, dD):
    """-tr(B D^{-1} dD D^{-1}) from a dense inverse."""
    M = Dinv @ (dD @ Dinv)
    return -np.sum(Bdiag * np.diag(M))
