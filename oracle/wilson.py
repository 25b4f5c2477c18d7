"""Oracle: the Wilson-Dirac operator (test infrastructure only).

Sec. 1 of the paper fixes D only as "12x12 spin-colour blocks per site with
nearest-neighbour coupling on a 4D torus"; it never writes the stencil out.
Reading taken here (standard hopping-parameter form, no clover term):

    (D psi)(x) = psi(x) - kappa * sum_{mu=0..3} [ (1 - g_mu) U_mu(x) psi(x+mu)
                                               + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu) ]

with g_mu the chiral gamma matrices of oracle.gamma, mu = 0..3 <-> x, y, z, t,
and a boundary factor bc[mu] (+1 periodic, -1 antiperiodic) on every hop that
wraps around the torus in direction mu.

Two independent forms are given: `apply` (whole-lattice array shifts) and
`sparse_matrix` (explicit per-site block assembly in a Python loop).  Tests
check them against each other, against gamma5-hermiticity, gauge covariance
and the free-field closed form.
"""
import numpy as np
import scipy.sparse as sp

from .gamma import GAMMA, ID4

# axis of direction mu in a (..., T, Z, Y, X, s, c) array
_AX = {0: -3, 1: -4, 2: -5, 3: -6}


def _shift(a, mu, step, bc):
    """Return b with b(x) = a(x + step*mu_hat) (step = +1 or -1), multiplied by
    bc[mu] wherever the hop wraps around the lattice."""
    ax = _AX[mu]
    L = a.shape[ax]
    b = np.roll(a, -step, axis=ax)
    if bc[mu] != 1:
        idx = [slice(None)] * a.ndim
        idx[ax] = L - 1 if step == 1 else 0   # sites whose neighbour wrapped
        b[tuple(idx)] *= bc[mu]
    return b


def _spin(g, psi):
    return np.einsum('st,...tc->...sc', g, psi)


def _colour(u, psi):
    return np.einsum('...ab,...sb->...sa', u, psi)


def hop(U, psi, bc):
    """H psi = sum_mu [(1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^+ psi(x-mu)].

    U: (4, T, Z, Y, X, 3, 3); psi: (..., T, Z, Y, X, 4, 3)."""
    out = np.zeros_like(psi)
    for mu in range(4):
        fwd = _colour(U[mu], _shift(psi, mu, +1, bc))
        out += _spin(ID4 - GAMMA[mu], fwd)
        # U_mu(x-mu)^+ psi(x-mu): shift both the link and the spinor back, the
        # wrap factor applied once (to the spinor)
        ub = np.roll(U[mu], 1, axis=_AX[mu])
        bwd = _colour(np.swapaxes(ub.conj(), -1, -2), _shift(psi, mu, -1, bc))
        out += _spin(ID4 + GAMMA[mu], bwd)
    return out


def apply(U, psi, kappa, bc):
    """D psi = psi - kappa H psi."""
    return psi - kappa * hop(U, psi, bc)


def apply_dagger(U, psi, kappa, bc):
    """D^+ psi, from the stencil with (1 -/+ g) swapped and kappa conjugated
    (kappa is real): D^+ = 1 - kappa sum [(1+g) U psi(x+mu) + (1-g) U^+ psi(x-mu)]."""
    out = np.zeros_like(psi)
    for mu in range(4):
        fwd = _colour(U[mu], _shift(psi, mu, +1, bc))
        out += _spin(ID4 + GAMMA[mu], fwd)
        ub = np.roll(U[mu], 1, axis=_AX[mu])
        bwd = _colour(np.swapaxes(ub.conj(), -1, -2), _shift(psi, mu, -1, bc))
        out += _spin(ID4 - GAMMA[mu], bwd)
    return psi - kappa * out


def site_index(dims, x, y, z, t):
    X, Y, Z, T = dims
    return x + X * (y + Y * (z + Z * t))


def sparse_matrix(U, kappa, bc):
    """D as an explicit n x n scipy CSR matrix, n = 12 V, dof index
    12*site + 3*spin + colour.  Assembled block by block in a loop over sites
    and directions (independent of `apply`)."""
    T, Z, Y, X = U.shape[1:5]
    dims = (X, Y, Z, T)
    V = X * Y * Z * T
    rows, cols, vals = [], [], []
    eye12 = np.eye(12)
    r12 = np.arange(12)
    for t in range(T):
        for z in range(Z):
            for y in range(Y):
                for x in range(X):
                    s = site_index(dims, x, y, z, t)
                    c = [x, y, z, t]
                    rows.append(12 * s + r12); cols.append(12 * s + r12)
                    vals.append(np.ones(12))
                    for mu in range(4):
                        L = dims[mu]
                        # forward neighbour
                        cf = list(c); cf[mu] = (c[mu] + 1) % L
                        sgn_f = bc[mu] if c[mu] == L - 1 else 1
                        blk = -kappa * sgn_f * np.kron(ID4 - GAMMA[mu], U[mu, t, z, y, x])
                        sf = site_index(dims, *cf)
                        rr, cc = np.nonzero(np.abs(blk) > 0)
                        rows.append(12 * s + rr); cols.append(12 * sf + cc); vals.append(blk[rr, cc])
                        # backward neighbour: link U_mu(x - mu) daggered
                        cb = list(c); cb[mu] = (c[mu] - 1) % L
                        sgn_b = bc[mu] if c[mu] == 0 else 1
                        ulink = U[mu, cb[3], cb[2], cb[1], cb[0]]
                        blk = -kappa * sgn_b * np.kron(ID4 + GAMMA[mu], ulink.conj().T)
                        sb = site_index(dims, *cb)
                        rr, cc = np.nonzero(np.abs(blk) > 0)
                        rows.append(12 * s + rr); cols.append(12 * sb + cc); vals.append(blk[rr, cc])
    del eye12
    rows = np.concatenate(rows); cols = np.concatenate(cols); vals = np.concatenate(vals)
    n = 12 * V
    # duplicates (lattice extent 2: x+mu == x-mu, or extent 1) are summed
    return sp.csr_matrix((vals.astype(np.complex128), (rows, cols)), shape=(n, n))


def gamma5_full(V):
    """gamma5 (x) 1_colour on every site, as a length-12V diagonal."""
    from .gamma import GAMMA5
    return np.tile(np.repeat(np.diag(GAMMA5).real, 3), V)


def timeslice_of_dof(dims):
    """Timeslice t of every dof (length 12 V)."""
    X, Y, Z, T = dims
    return np.repeat(np.arange(T), X * Y * Z * 12)
