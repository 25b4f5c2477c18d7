"""Pins of the connected-correlator oracle (Sec. 4, Eqs. 16-20, L = 2)."""
import numpy as np
import pytest

import synth
from oracle import connected, freefield, multigrid, solver, wilson

BC = (1, 1, 1, -1)


@pytest.fixture(scope='module')
def setup():
    dims, agg, nv = (2, 2, 2, 4), (2, 2, 2, 2), 3
    U = synth.gauge_field(dims, 0.4, 1020)
    D = wilson.sparse_matrix(U, 0.12, BC)
    P = multigrid.prolongator(synth.test_vectors(dims, nv, 21), dims, agg)
    Dinv = solver.dense_inverse(D)
    Dcinv = solver.dense_inverse(multigrid.coarse_operator(D, P))
    return dims, D, P, Dinv, Dcinv


def test_correlator_is_frobenius_norm_of_propagator_blocks(setup):
    """Eq. 16 with gamma5-hermiticity D^{-1}(t', t+t') = g5 D^{-1}(t+t', t')^dag g5:
    G(t) = (1/T) sum_t' ||D^{-1}(t+t', t')||_F^2, real and positive."""
    dims, D, P, Dinv, Dcinv = setup
    T = dims[3]
    ts = wilson.timeslice_of_dof(dims)
    ref = np.array([sum(np.linalg.norm(Dinv[np.ix_(ts == (t + tp) % T, ts == tp)]) ** 2 for tp in range(T)) / T
                    for t in range(T)])
    G = connected.correlator_exact(Dinv, Dinv, dims)
    assert np.abs(G - ref).max() < 1e-13 * ref.max() and np.all(ref > 0)


@pytest.mark.parametrize("dims,bc", [((2, 2, 2, 4), (1, 1, 1, -1)), ((4, 2, 2, 6), (1, 1, 1, 1))])
def test_free_field_matches_momentum_sum(dims, bc):
    """Unit links: translation invariance makes Eq. 16 equal to
    X*Y*Z times the point-source correlator sum_x ||D^{-1}(x; 0)||_F^2, which
    the free-field oracle computes from the momentum-space propagator
    (independent of the assembled operator)."""
    U = synth.unit_gauge(dims)
    Dinv = solver.dense_inverse(wilson.sparse_matrix(U, 0.11, bc))
    G = connected.correlator_exact(Dinv, Dinv, dims)
    ref = dims[0] * dims[1] * dims[2] * freefield.pion_correlator(dims, 0.11, bc)
    assert np.abs(G.imag).max() < 1e-12 * ref.max()
    assert np.abs(G.real - ref).max() < 1e-11 * ref.max()


def test_level_operators_gamma5_hermitian_and_telescoping(setup):
    """B_1 + B_2 = D^{-1} (Eq. 10) and both are gamma5-hermitian (P keeps the
    chirality halves apart), and sum_ij G_ij = G (Eq. 19)."""
    dims, D, P, Dinv, Dcinv = setup
    B1, B2 = connected.level_operators(Dinv, P.toarray(), Dcinv)
    assert np.abs(B1 + B2 - Dinv).max() < 1e-13 * np.abs(Dinv).max()
    g5 = wilson.gamma5_full(int(np.prod(dims)))
    for B in (B1, B2):
        assert np.abs(g5[:, None] * B.conj().T * g5[None, :] - B).max() < 1e-12 * np.abs(B).max()
    G = connected.correlator_exact(Dinv, Dinv, dims)
    Gs = sum(connected.correlator_exact(Bi, Bj, dims) for Bi in (B1, B2) for Bj in (B1, B2))
    assert np.abs(Gs - G).max() < 1e-12 * np.abs(G).max()


def test_estimator_expectation_is_exact(setup):
    """Replacing the noise by every unit vector of the source timeslice (the
    estimator's expectation, E[eta eta^dag] = 1) reproduces every G_ij(t)
    of the trace definition; the Rademacher samples average towards it."""
    dims, D, P, Dinv, Dcinv = setup
    T = dims[3]
    Pd = P.toarray()
    B1, B2 = connected.level_operators(Dinv, Pd, Dcinv)
    ts = wilson.timeslice_of_dof(dims)
    n = Dinv.shape[0]
    ys = {1: B1, 2: B2}
    for (i, j) in ((1, 1), (1, 2), (2, 1), (2, 2)):
        ref = connected.correlator_exact(ys[i], ys[j], dims)
        est = np.zeros(T, np.complex128)
        for tp in range(T):
            for k in np.where(ts == tp)[0]:
                e = np.zeros(n); e[k] = 1.0
                yi, yj = ys[i] @ e, ys[j] @ e
                for t in range(T):
                    m = ts == (t + tp) % T
                    est[t] += np.vdot(yj[m], yi[m]) / T
        assert np.abs(est - ref).max() < 1e-12 * np.abs(ref).max(), (i, j)
    S1, S2 = connected.samples(lambda v: Dinv @ v, lambda v: Dcinv @ v, P, dims, 3, 64, 64)
    G11 = connected.correlator_exact(B1, B1, dims)
    G22 = connected.correlator_exact(B2, B2, dims)
    sd1 = S1[:, 0].std(axis=0) / np.sqrt(64)
    sd2 = S2.std(axis=0) / np.sqrt(64)
    assert np.all(np.abs(S1[:, 0].mean(0) - G11) < 5 * sd1 + 1e-12)
    assert np.all(np.abs(S2.mean(0) - G22) < 5 * sd2 + 1e-12)
    # (2,1) is the conjugate of (1,2) sample by sample
    assert np.abs(S1[:, 2] - S1[:, 1].conj()).max() < 1e-14 * np.abs(S1).max()


def test_estimate_combines_pinned_means_and_variances(setup):
    """estimate(): the pair means and variances are the pinned sample mean and
    variance of the mean; the total's variance adds the independent levels."""
    from oracle import estimators
    dims, D, P, Dinv, Dcinv = setup
    S1, S2 = connected.samples(lambda v: Dinv @ v, lambda v: Dcinv @ v, P, dims, 9, 5, 7)
    G, var = connected.estimate(S1, S2)
    for k, S in enumerate((S1[:, 0], S1[:, 1], S1[:, 2], S2)):
        m, v, _, _ = estimators.mean_and_variance(S)
        assert np.allclose(G[k], m, rtol=1e-14, atol=0) and np.allclose(var[k], v / S.shape[0], rtol=1e-12)
    m1, v1, _, _ = estimators.mean_and_variance(S1[:, :3].sum(1))
    m2, v2, _, _ = estimators.mean_and_variance(S2)
    assert np.allclose(G[4], m1 + m2, rtol=1e-14) and np.allclose(var[4], v1 / 5 + v2 / 7, rtol=1e-12)
    mp, vp, _, _ = estimators.mean_and_variance(S1.sum(1))
    assert np.allclose(G[5], mp, rtol=1e-14) and np.allclose(var[5], vp / 5, rtol=1e-12)


def test_plain_sample_is_the_undecomposed_estimator(setup):
    """The four level-1 columns sum to |D^{-1} eta|^2 on the source-shifted
    timeslices: the plain estimator of Eq. 16, sample by sample."""
    dims, D, P, Dinv, Dcinv = setup
    T = dims[3]
    from oracle import noise
    S1, _ = connected.samples(lambda v: Dinv @ v, lambda v: Dcinv @ v, P, dims, 4, 2, 2)
    ts = wilson.timeslice_of_dof(dims)
    for i in range(2):
        eta = noise.rademacher(4, i, Dinv.shape[0])
        ref = np.zeros(T, np.complex128)
        for tp in range(T):
            y = Dinv @ np.where(ts == tp, eta, 0).astype(complex)
            for t in range(T):
                m = ts == (t + tp) % T
                ref[t] += np.vdot(y[m], y[m]) / T
        assert np.abs(S1[i].sum(0) - ref).max() < 1e-12 * np.abs(ref).max()
