"""Pins of the two-level hierarchy (Sec. 2, Eqs. 7-12)."""
import numpy as np
import pytest

import synth
from oracle import estimators, multigrid, solver, wilson

BC_AP = (1, 1, 1, -1)


@pytest.fixture(scope='module')
def mg():
    dims, agg, nv = (4, 4, 4, 4), (2, 2, 2, 2), 4
    U = synth.gauge_field(dims, 0.3, 1004)
    D = wilson.sparse_matrix(U, 0.12, BC_AP)
    tv = synth.test_vectors(dims, nv, 77)
    P = multigrid.prolongator(tv, dims, agg)
    Dc = multigrid.coarse_operator(D, P)
    Dinv = solver.dense_inverse(D)
    Dcinv = solver.dense_inverse(Dc)
    return dims, agg, nv, U, D, P, Dc, Dinv, Dcinv


def test_orthonormal(mg):
    P = mg[5]
    PP = (P.conj().T @ P).toarray()
    assert np.abs(PP - np.eye(PP.shape[0])).max() < 1e-14


def test_oblique_projector_is_projector(mg):
    """Eq. 8: Pi = P D_c^{-1} P^dag D is idempotent (needs D_c = P^dag D P)."""
    dims, agg, nv, U, D, P, Dc, Dinv, Dcinv = mg
    Pd = P.toarray()
    Pi = Pd @ Dcinv @ (Pd.conj().T @ D.toarray())
    assert np.abs(Pi @ Pi - Pi).max() < 1e-11 * np.abs(Pi).max()


def test_telescoping(mg):
    """Eq. 11 with L = 2: tr(M_1) + tr(D_c^{-1}) = tr(D^{-1})."""
    dims, agg, nv, U, D, P, Dc, Dinv, Dcinv = mg
    Pd = P.toarray()
    M = Dinv - Pd @ Dcinv @ Pd.conj().T
    assert abs(np.trace(M) + np.trace(Dcinv) - np.trace(Dinv)) < 1e-12 * abs(np.trace(Dinv))


def test_unitary_prolongator_gives_zero_difference():
    """With one-site aggregates and 6 test vectors P is unitary, so
    M_1 = D^{-1} - P (P^dag D P)^{-1} P^dag vanishes (Eq. 10)."""
    dims = (2, 2, 2, 4)
    U = synth.gauge_field(dims, 0.5, 9)
    D = wilson.sparse_matrix(U, 0.13, BC_AP)
    P = multigrid.prolongator(synth.test_vectors(dims, 6, 1), dims, (1, 1, 1, 1))
    Dc = multigrid.coarse_operator(D, P)
    Pd = P.toarray()
    M = solver.dense_inverse(D) - Pd @ solver.dense_inverse(Dc) @ Pd.conj().T
    assert np.abs(M).max() < 1e-11


def test_coarse_gamma5_hermiticity(mg):
    dims, agg, nv, U, D, P, Dc, Dinv, Dcinv = mg
    g5c = multigrid.gamma5_coarse(nv, P.shape[1] // (2 * nv))
    Dcd = Dc.toarray()
    assert np.abs(Dcd.conj().T - g5c[:, None] * Dcd * g5c[None, :]).max() < 1e-13


def test_coarse_nine_point_sparsity():
    """D_c couples a coarse site only to itself and its 8 nearest neighbours."""
    dims, agg, nv = (6, 6, 6, 6), (2, 2, 2, 2), 2
    U = synth.gauge_field(dims, 0.5, 3)
    D = wilson.sparse_matrix(U, 0.13, BC_AP)
    P = multigrid.prolongator(synth.test_vectors(dims, nv, 2), dims, agg)
    Dc = multigrid.coarse_operator(D, P).tocoo()
    cd = multigrid.coarse_dims(dims, agg)
    k = 2 * nv
    def coords(c):
        out = []
        for L in cd:
            out.append(c % L); c //= L
        return np.array(out)
    a, b = coords(Dc.row // k), coords(Dc.col // k)
    diff = np.abs(a - b)
    diff = np.minimum(diff, np.array(cd)[:, None] - diff)
    assert diff.sum(axis=0).max() == 1
    assert len(set(zip(Dc.row // k, Dc.col // k))) == np.prod(cd) * 9


def test_mlmc_unbiased_and_level_variances(mg):
    dims, agg, nv, U, D, P, Dc, Dinv, Dcinv = mg
    Pd = P.toarray()
    N1, N2 = 96, 256
    X1, X2 = estimators.mlmc2(lambda v: Dinv @ v, lambda v: Dcinv @ v, P, dims, 2004, N1, N2, False)
    _, _, m1, v1 = estimators.mean_and_variance(X1)
    _, _, m2, v2 = estimators.mean_and_variance(X2)
    M = Dinv - Pd @ Dcinv @ Pd.conj().T
    V1 = estimators.hutchinson_variance(M)
    V2 = estimators.hutchinson_variance(Dcinv)
    assert abs(m1 - np.trace(M)) < 5 * np.sqrt(V1 / N1)
    assert abs(m2 - np.trace(Dcinv)) < 5 * np.sqrt(V2 / N2)
    assert 0.6 < v1 / V1 < 1.4 and 0.7 < v2 / V2 < 1.3
    total = m1 + m2
    assert abs(total - np.trace(Dinv)) < 5 * np.sqrt(V1 / N1 + V2 / N2)
