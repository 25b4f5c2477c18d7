"""Oracle: aggregation-based two-level hierarchy (test infrastructure only).

Sec. 2: R = P^dagger with P^dagger P = I, and the Galerkin coarse operator
D_c = P^dagger D P (Eq. 7).  The paper delegates the construction to the
DD-alpha-AMG setup; reading taken here (the usual aggregation scheme):
  * the fine lattice is cut into aggregates of agg[mu] sites per direction
    (4^4 in the large workloads);
  * every test vector is restricted to each aggregate and to each chirality
    half (gamma5 = +1: spins 0, 1; gamma5 = -1: spins 2, 3);
  * the restricted vectors of one (aggregate, half) are orthonormalised by
    modified Gram-Schmidt in test-vector order.
Coarse dof index = 2*nv*X_c + nv*h + k (coarse site X_c lexicographic, x fastest;
half h; test vector k).
"""
import numpy as np
import scipy.sparse as sp


def coarse_dims(dims, agg):
    for L, a in zip(dims, agg):
        if L % a:
            raise ValueError('aggregate size must divide the lattice extent')
    return tuple(L // a for L, a in zip(dims, agg))


def aggregate_rows(dims, agg):
    """For each (coarse site, half): the sorted fine dof indices it owns.
    Returns an int array (Vc, 2, m) with m = 6 * prod(agg)."""
    X, Y, Z, T = dims
    cd = coarse_dims(dims, agg)
    Vc = int(np.prod(cd))
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing='ij')
    site = (x + X * (y + Y * (z + Z * t))).reshape(-1)
    csite = ((x // agg[0]) + cd[0] * ((y // agg[1]) + cd[1] * ((z // agg[2]) + cd[2] * (t // agg[3])))).reshape(-1)
    rows = []
    for c in range(Vc):
        sites = np.sort(site[csite == c])
        per = []
        for h in range(2):
            d = (12 * sites[:, None] + 3 * (2 * h) + np.arange(6)[None, :]).reshape(-1)
            per.append(np.sort(d))
        rows.append(per)
    return np.array(rows)


def mgs(A):
    """Modified Gram-Schmidt on the columns of A (in column order)."""
    Q = np.array(A, dtype=np.complex128, copy=True)
    for k in range(Q.shape[1]):
        for j in range(k):
            Q[:, k] -= np.vdot(Q[:, j], Q[:, k]) * Q[:, j]
        Q[:, k] /= np.linalg.norm(Q[:, k])
    return Q


def prolongator(tv, dims, agg):
    """P as scipy CSR (12V x 2 nv Vc) from test vectors tv (nv, T, Z, Y, X, 4, 3)."""
    nv = tv.shape[0]
    flat = tv.reshape(nv, -1)
    rows = aggregate_rows(dims, agg)
    Vc = rows.shape[0]
    n = flat.shape[1]
    R, C, Vals = [], [], []
    for c in range(Vc):
        for h in range(2):
            r = rows[c, h]
            Q = mgs(flat[:, r].T)                # (m, nv)
            for k in range(nv):
                R.append(r); C.append(np.full(r.shape, 2 * nv * c + nv * h + k)); Vals.append(Q[:, k])
    return sp.csr_matrix((np.concatenate(Vals), (np.concatenate(R), np.concatenate(C))),
                         shape=(n, 2 * nv * Vc))


# Test vectors (Sec. 2: the near-null space that P must capture; the paper takes
# them from the DD-alpha-AMG setup).  Reading: N_v inverse iterations from
# Rademacher starts -- start k is the noise vector of sample TV_STREAM + k
# (Eq. 1's generator, a stream of its own), and each step replaces v by
# D^{-1} v / ||D^{-1} v||, the 2-norm taken over the whole lattice.  The solve
# is FP64 BiCGStab on the full operator.
TV_STREAM = 1 << 22


def test_vectors(apply_D, dims, nv, iters, seed, tol=1e-12):
    """(nv, T, Z, Y, X, 4, 3) complex128: `iters` normalised inverse iterations
    of the Rademacher starts of samples TV_STREAM + k, k < nv (iters = 0: the
    starts themselves, unnormalised)."""
    from .noise import rademacher
    from .solver import bicgstab
    X, Y, Z, T = dims
    n = 12 * X * Y * Z * T
    shape = (T, Z, Y, X, 4, 3)
    out = np.empty((nv,) + shape, np.complex128)
    for k in range(nv):
        v = rademacher(seed, TV_STREAM + k, n).astype(np.complex128).reshape(shape)
        for _ in range(iters):
            x, _, _ = bicgstab(apply_D, v, tol=tol)
            v = x / np.linalg.norm(x)
        out[k] = v
    return out


def coarse_operator(Dmat, P):
    """Eq. 7: D_c = P^dagger D P (sparse)."""
    Ph = P.conj().T.tocsr()
    return (Ph @ (Dmat @ P)).tocsr()


def gamma5_coarse(nv, Vc):
    """gamma5 on the coarse space: +1 on half 0, -1 on half 1 of every coarse site."""
    return np.tile(np.concatenate([np.ones(nv), -np.ones(nv)]), Vc)


# ---- a third level (Sec. 2 with L = 3; the hierarchy of the paper's Table 2) --
# The coarse space is aggregated again: coarse sites (coarse extents cd, coarse
# dof index 2 nv X + nv h + k) are grouped into aggregates of agg2 coarse sites
# per direction, every level-2 test vector is restricted to each aggregate and
# chirality half h (the coarse dofs of half h keep the chirality of the fine
# spins they came from), and the pieces of one (aggregate, half) are
# orthonormalised by modified Gram-Schmidt in test-vector order.  Level-3 dof
# index = 2 nv2 Xcc + nv2 h + k.  D_3 = P_2^dag D_c P_2 (Eq. 7 with l = 2).

def aggregate_rows_coarse(cd, agg2, nv):
    """For each (level-3 site, half): the sorted level-2 dof indices it owns.
    Returns an int array (Vcc, 2, m) with m = nv * prod(agg2)."""
    ccd = coarse_dims(cd, agg2)
    Vcc = int(np.prod(ccd))
    t, z, y, x = np.meshgrid(*[np.arange(L) for L in cd[::-1]], indexing='ij')
    site = (x + cd[0] * (y + cd[1] * (z + cd[2] * t))).reshape(-1)
    csite = ((x // agg2[0]) + ccd[0] * ((y // agg2[1]) + ccd[1] * ((z // agg2[2]) + ccd[2] * (t // agg2[3])))).reshape(-1)
    rows = []
    for c in range(Vcc):
        sites = np.sort(site[csite == c])
        rows.append([np.sort((2 * nv * sites[:, None] + nv * h + np.arange(nv)[None, :]).reshape(-1)) for h in range(2)])
    return np.array(rows)


def prolongator_coarse(tv2, cd, agg2, nv):
    """P_2 as scipy CSR (2 nv Vc x 2 nv2 Vcc) from level-2 test vectors
    tv2 (nv2, 2 nv Vc) (coarse dof order)."""
    nv2 = tv2.shape[0]
    rows = aggregate_rows_coarse(cd, agg2, nv)
    Vcc = rows.shape[0]
    n = tv2.shape[1]
    R, C, Vals = [], [], []
    for c in range(Vcc):
        for h in range(2):
            r = rows[c, h]
            Q = mgs(tv2[:, r].T)
            for k in range(nv2):
                R.append(r); C.append(np.full(r.shape, 2 * nv2 * c + nv2 * h + k)); Vals.append(Q[:, k])
    return sp.csr_matrix((np.concatenate(Vals), (np.concatenate(R), np.concatenate(C))), shape=(n, 2 * nv2 * Vcc))
