"""Pins of the oracle's Wilson-Dirac operator (Sec. 1: 12x12 blocks, 4D torus)
against things the operator's definition fixes independently of the code:
two independent constructions, gamma algebra, gamma5-hermiticity, gauge
covariance and the free-field closed form."""
import numpy as np
import pytest

import synth
from oracle import freefield, gamma, solver, wilson

BC_AP = (1, 1, 1, -1)


def test_gamma_algebra():
    g = gamma.GAMMA
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)
        for n in range(4):
            ac = g[m] @ g[n] + g[n] @ g[m]
            assert np.allclose(ac, 2 * (m == n) * np.eye(4))
    assert np.allclose(gamma.GAMMA5, np.diag([1, 1, -1, -1]))


def test_gauge_is_su3():
    U = synth.gauge_field((4, 2, 2, 6), 0.5, 7)
    UU = np.einsum('...ba,...bc->...ac', U.conj(), U)
    assert np.abs(UU - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 2, 6), (3, 2, 1, 4)])
def test_stencil_matches_assembled_matrix(dims):
    U = synth.gauge_field(dims, 0.5, 11)
    psi = synth.spinors(dims, 2, 12)
    D = wilson.sparse_matrix(U, 0.13, BC_AP)
    y1 = wilson.apply(U, psi, 0.13, BC_AP).reshape(2, -1)
    y2 = np.stack([D @ p for p in psi.reshape(2, -1)])
    assert np.abs(y1 - y2).max() < 1e-13 * np.abs(y2).max()
    # the adjoint stencil is the conjugate transpose of the assembled matrix
    z1 = wilson.apply_dagger(U, psi, 0.13, BC_AP).reshape(2, -1)
    z2 = np.stack([D.conj().T @ p for p in psi.reshape(2, -1)])
    assert np.abs(z1 - z2).max() < 1e-13 * np.abs(z2).max()


def test_gamma5_hermiticity():
    """<phi, D psi> = <g5 D g5 phi, psi>, i.e. D^dag = g5 D g5."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.5, 3)
    phi, psi = synth.spinors(dims, 2, 4)
    g5 = np.diag(gamma.GAMMA5)[:, None]
    lhs = np.vdot(phi, wilson.apply(U, psi, 0.12, BC_AP))
    rhs = np.vdot(g5 * wilson.apply(U, g5 * phi, 0.12, BC_AP), psi)
    assert abs(lhs - rhs) < 1e-14 * abs(lhs) * 10


def test_gauge_covariance():
    """D[U^g] (g psi) = g (D[U] psi) with U^g_mu(x) = g(x) U_mu(x) g(x+mu)^dag.
    Fails for a wrong link orientation in either hop."""
    dims = (4, 2, 4, 6)
    U = synth.gauge_field(dims, 0.5, 5)
    g = synth.gauge_field(dims, 1.0, 6)[0]          # one SU(3) matrix per site
    Ug = np.empty_like(U)
    ax = {0: -3, 1: -4, 2: -5, 3: -6}
    for mu in range(4):
        gp = np.roll(g, -1, axis=ax[mu] + 0)        # g(x+mu) on (T,Z,Y,X,3,3)
        Ug[mu] = g @ U[mu] @ np.swapaxes(gp.conj(), -1, -2)
    psi = synth.spinors(dims, 1, 8)[0]
    gpsi = np.einsum('...ab,...sb->...sa', g, psi)
    lhs = wilson.apply(Ug, gpsi, 0.13, BC_AP)
    rhs = np.einsum('...ab,...sb->...sa', g, wilson.apply(U, psi, 0.13, BC_AP))
    assert np.abs(lhs - rhs).max() < 1e-13


@pytest.mark.parametrize("bc", [(1, 1, 1, -1), (1, 1, 1, 1)])
def test_free_field_trace(bc):
    """U = 1: tr D^{-1} = 12 sum_p a/(a^2+|b|^2) (momentum sum) vs dense LU."""
    dims = (4, 4, 4, 4)
    D = wilson.sparse_matrix(synth.unit_gauge(dims), 0.12, bc)
    Dinv = solver.dense_inverse(D)
    ex = np.trace(Dinv)
    cf = freefield.trace_inverse(dims, 0.12, bc)
    assert abs(ex - cf) < 1e-12 * abs(cf)
    # tr[g5 D^{-1}(t,t)] vanishes for the free field
    assert np.abs(solver.exact_traces(Dinv, dims, True)).max() < 1e-12


def test_free_field_point_propagator():
    """Columns of D^{-1} for a source at the origin vs the momentum sum, and
    the pion correlator C(t) built from them."""
    dims = (2, 4, 2, 6)
    kappa = 0.124
    D = wilson.sparse_matrix(synth.unit_gauge(dims), kappa, BC_AP)
    Dinv = solver.dense_inverse(D)
    S = freefield.point_propagator(dims, kappa, BC_AP)      # (T,Z,Y,X,4,4)
    X, Y, Z, T = dims
    cols = Dinv[:, :12].reshape(T, Z, Y, X, 4, 3, 4, 3)    # (x, s, a; s', a')
    expect = np.einsum('...st,ab->...satb', S, np.eye(3))
    assert np.abs(cols - expect).max() < 1e-12
    C = freefield.pion_correlator(dims, kappa, BC_AP)
    C2 = (np.abs(cols) ** 2).reshape(T, -1).sum(axis=1)
    assert np.allclose(C, C2, rtol=1e-12)


def test_bicgstab_matches_dense():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1001)
    D = wilson.sparse_matrix(U, 0.12, BC_AP)
    b = synth.spinors(dims, 1, 3).reshape(-1)
    x, it, res = solver.bicgstab(lambda v: wilson.apply(U, v.reshape(synth.spinors(dims, 1, 0).shape[1:]), 0.12, BC_AP), b, tol=1e-12)
    assert res < 1e-11
    xd = np.linalg.solve(D.toarray(), b)
    assert np.linalg.norm(x - xd) < 1e-10 * np.linalg.norm(xd)
