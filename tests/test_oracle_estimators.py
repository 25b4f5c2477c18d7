"""Pins of the oracle estimators: exact enumeration over all Rademacher sign
patterns (the variance formula of Eq. 4 and its probing analogue), the exact
probing limit, and statistical unbiasedness against dense-LU traces."""
import itertools

import numpy as np
import pytest

import synth
from oracle import coloring, estimators, solver, wilson

BC_AP = (1, 1, 1, -1)


def _signs(n):
    return np.array(list(itertools.product((-1.0, 1.0), repeat=n)))


def test_hutchinson_variance_by_enumeration():
    """Over all 2^n sign vectors: mean of eta^T A eta = tr A exactly and the
    variance equals 1/2 ||offdiag(A + A^T)||_F^2 (Eq. 4), for complex A."""
    rng = np.random.default_rng(0)
    n = 10
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    E = _signs(n)
    X = np.einsum('ij,jk,ik->i', E, A, E)
    assert abs(X.mean() - np.trace(A)) < 1e-12
    var = np.mean(np.abs(X - np.trace(A)) ** 2)
    assert abs(var - estimators.hutchinson_variance(A)) < 1e-10 * var


def test_probing_variance_by_enumeration():
    rng = np.random.default_rng(1)
    n = 12
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    groups = rng.integers(0, 3, n)
    E = _signs(n)
    X = np.zeros(len(E), complex)
    for g in range(3):
        m = groups == g
        Eg = E * m
        X += np.einsum('ij,jk,ik->i', Eg, A, Eg)
    assert abs(X.mean() - np.trace(A)) < 1e-12
    var = np.mean(np.abs(X - np.trace(A)) ** 2)
    assert abs(var - estimators.probing_variance(A, groups)) < 1e-10 * var
    # a single group reduces to the Hutchinson formula
    assert abs(estimators.probing_variance(A, np.zeros(n)) - estimators.hutchinson_variance(A)) < 1e-10


@pytest.fixture(scope='module')
def small():
    dims = (2, 4, 2, 6)
    U = synth.gauge_field(dims, 0.3, 1001)
    D = wilson.sparse_matrix(U, 0.12, BC_AP)
    Dinv = solver.dense_inverse(D)
    return dims, U, D, Dinv


def test_probing_exact_limit(small):
    """Every site its own colour and full dilution: every sample gives the
    exact per-timeslice trace (probing is then deterministic)."""
    dims, U, D, Dinv = small
    V = int(np.prod(dims))
    col = np.arange(V, dtype=np.int32)
    ex = solver.exact_traces(Dinv, dims, True)
    X = estimators.probing(lambda v: Dinv @ v, dims, 2001, 2, True, col, V, 12)
    assert np.abs(X - ex[None]).max() < 1e-12 * np.abs(ex).max() + 1e-14


def test_probing_variance_matches_closed_form(small):
    """Empirical variance of the probing x dilution total over 400 samples vs
    the closed form, within the statistical spread."""
    dims, U, D, Dinv = small
    nc, sigma = coloring.search(dims, 1)
    col = coloring.colors(dims, sigma, nc)
    masks = estimators.probing_masks(col, nc, 12)
    groups = np.argmax(masks, axis=0)
    A = Dinv * wilson.gamma5_full(int(np.prod(dims)))[:, None]
    N = 400
    X = estimators.probing(lambda v: Dinv @ v, dims, 5, N, True, col, nc, 12)
    _, _, mt, vt = estimators.mean_and_variance(X)
    Vf = estimators.probing_variance(A, groups)
    assert abs(mt - np.trace(A)) < 5 * np.sqrt(Vf / N)
    assert 0.7 < vt / Vf < 1.3


def test_hutchinson_statistics_4x4x4x4():
    """Hutchinson on the 4^4 lattice of the smallest workload: mean within
    5 sigma of the exact trace, sample variance near Eq. 4."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1001)
    D = wilson.sparse_matrix(U, 0.12, BC_AP)
    Dinv = solver.dense_inverse(D)
    N = 256
    X = estimators.hutchinson(lambda v: Dinv @ v, dims, 2001, N, False)
    _, var_t, mt, vt = estimators.mean_and_variance(X)
    ex = np.trace(Dinv)
    Vf = estimators.hutchinson_variance(Dinv)
    assert abs(mt - ex) < 5 * np.sqrt(Vf / N)
    assert 0.7 < vt / Vf < 1.3
    # time-diluted gamma5 estimator is unbiased per timeslice
    Xt = estimators.hutchinson(lambda v: Dinv @ v, dims, 2001, 64, True, time_dilution=True)
    ext = solver.exact_traces(Dinv, dims, True)
    m, v, _, _ = estimators.mean_and_variance(Xt)
    assert np.all(np.abs(m - ext) < 6 * np.sqrt(v / 64) + 1e-12)


def test_gamma5_trace_is_real(small):
    """gamma5-hermiticity makes tr[g5 D^{-1}(t,t)] real."""
    dims, U, D, Dinv = small
    ext = solver.exact_traces(Dinv, dims, True)
    assert np.abs(ext.imag).max() < 1e-12 * np.abs(ext).max()


def test_mean_and_variance_special_case():
    x = np.random.default_rng(3).standard_normal((50, 4))
    m, v, mt, vt = estimators.mean_and_variance(x)
    assert np.allclose(m, x.mean(0)) and np.allclose(v, x.var(0, ddof=1))
    assert np.isclose(vt, x.sum(1).var(ddof=1))
