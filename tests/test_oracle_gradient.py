"""Pins of the derivative formulas: finite differences of exact dense traces,
the definition dX = -w^dag dD z, and the exact probing limit."""
import numpy as np
import scipy.linalg as sla

import synth
from oracle import estimators, gradient, solver, wilson

BC_AP = (1, 1, 1, -1)
DIMS = (2, 4, 2, 6)


def _expm_links(T, h):
    return np.array([sla.expm(1j * h * t) for t in T.reshape(-1, 3, 3)]).reshape(T.shape)


def test_exact_derivative_vs_finite_difference():
    U = synth.gauge_field(DIMS, 0.5, 5)
    T = synth.su3_algebra(DIMS, 6)
    kappa = 0.125
    V = int(np.prod(DIMS))
    g5 = wilson.gamma5_full(V)
    def trace(h):
        Uh = np.einsum('...ab,...bc->...ac', _expm_links(T, h), U)
        Dinv = solver.dense_inverse(wilson.sparse_matrix(Uh, kappa, BC_AP))
        return np.sum(g5 * np.diag(Dinv))
    h = 1e-5
    fd = (trace(h) - trace(-h)) / (2 * h)
    Dinv = solver.dense_inverse(wilson.sparse_matrix(U, kappa, BC_AP))
    Delta = 1j * np.einsum('...ab,...bc->...ac', T, U)
    an = gradient.exact_derivative(Dinv, g5, gradient.hopping_derivative(Delta, kappa, BC_AP))
    assert abs(fd - an) < 1e-6 * abs(an)


def test_force_matches_definition():
    """sum tr(Delta G) + conj(tr(Delta H)) == -w^dag dD z for random w, z, Delta."""
    U = synth.gauge_field(DIMS, 0.5, 7)
    w = synth.spinors(DIMS, 2, 8)
    z = synth.spinors(DIMS, 2, 9)
    rng = np.random.default_rng(0)
    Delta = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    kappa = 0.13
    G, H = gradient.link_force(w, z, kappa, BC_AP)
    got = gradient.directional(G, H, Delta)
    dD = gradient.hopping_derivative(Delta, kappa, BC_AP)
    want = -sum(np.vdot(w[i].reshape(-1), dD @ z[i].reshape(-1)) for i in range(2))
    assert abs(got - want) < 1e-12 * abs(want)


def test_probing_limit_gives_exact_gradient():
    """n_c = V with full dilution: the sum of per-vector forces equals the exact
    derivative -tr(g5 D^{-1} dD D^{-1})."""
    U = synth.gauge_field(DIMS, 0.5, 10)
    kappa = 0.125
    V = int(np.prod(DIMS))
    g5 = wilson.gamma5_full(V)
    D = wilson.sparse_matrix(U, kappa, BC_AP)
    Dinv = solver.dense_inverse(D)
    from oracle import noise
    eta = noise.rademacher(1, 0, 12 * V)
    shape = (1,) + synth.spinors(DIMS, 1, 0).shape[1:]
    zs, ws = [], []
    for j in range(12 * V):
        v = np.zeros(12 * V, complex); v[j] = eta[j]
        zs.append(Dinv @ v)
        ws.append(Dinv.conj().T @ (g5 * v))
    zs = np.array(zs).reshape((-1,) + shape[1:])
    ws = np.array(ws).reshape((-1,) + shape[1:])
    G, H = gradient.link_force(ws, zs, kappa, BC_AP)
    T = synth.su3_algebra(DIMS, 11)
    Delta = 1j * np.einsum('...ab,...bc->...ac', T, U)
    est = gradient.directional(G, H, Delta)
    ex = gradient.exact_derivative(Dinv, g5, gradient.hopping_derivative(Delta, kappa, BC_AP))
    assert abs(est - ex) < 1e-10 * abs(ex)


def test_kappa_derivative():
    U = synth.gauge_field(DIMS, 0.5, 12)
    V = int(np.prod(DIMS))
    g5 = wilson.gamma5_full(V)
    v = synth.spinors(DIMS, 1, 13).reshape(-1)
    def X(k):
        return np.vdot(v, g5 * np.linalg.solve(wilson.sparse_matrix(U, k, BC_AP).toarray(), v))
    k, h = 0.125, 1e-6
    fd = (X(k + h) - X(k - h)) / (2 * h)
    D = wilson.sparse_matrix(U, k, BC_AP).toarray()
    z = np.linalg.solve(D, v)
    w = np.linalg.solve(D.conj().T, g5 * v)
    an = (np.vdot(w, z) - X(k)) / k
    assert abs(fd - an) < 1e-6 * abs(an)
