"""Parity of trace_estimate (noise, solves, contractions) with the oracle on identical
seeded noise: per-sample values X_i(t) element by element.

Tolerance reading: solves at 1e-12 on both sides bound the error of one
quadratic form by ~|eta| |x - x*|, not by |X|, so the comparison is
|X_gpu - X_oracle| <= 1e-8 * max(|X_oracle|, mean_i sum_t |X_i(t)|)."""
import numpy as np
import pytest

import synth
from oracle import coloring, estimators, solver, wilson
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu
BC = (1, 1, 1, -1)


def _close(gpu, ref):
    scale = max(np.abs(ref).max(), np.abs(ref).sum(axis=1).mean())
    assert np.abs(gpu - ref).max() <= 1e-8 * scale, np.abs(gpu - ref).max() / scale


@pytest.fixture(scope='module')
def tiny():
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1001)
    Dinv = solver.dense_inverse(wilson.sparse_matrix(U, 0.12, BC))
    return dims, U, 0.12, Dinv


@pytest.mark.parametrize("gamma5", [0, 1])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_hutchinson_4x4x4x4(tiny, gamma5, prec):
    """The smallest workload: 4^4, kappa 0.12, N = 64 Rademacher vectors."""
    from paper_2607_05157_b300 import Context, trace_estimate, WD_HUTCH
    dims, U, kappa, Dinv = tiny
    ctx = Context(dims, U, kappa, BC)
    r = trace_estimate(ctx.h, WD_HUTCH, 1, 64, dims[3], seed=2001, op=gamma5, prec=prec, tol=1e-12,
                       with_samples=True)
    ref = estimators.hutchinson(lambda v: Dinv @ v, dims, 2001, 64, bool(gamma5))
    _close(r['samples'], ref)
    m, v, mt, vt = estimators.mean_and_variance(ref)
    assert np.allclose(r['estimate'], m, rtol=1e-8, atol=1e-8 * np.abs(ref).sum(1).mean())
    assert abs(r['total'] - mt) <= 1e-8 * np.abs(ref).sum(1).mean()
    assert np.allclose(r['var'], v, rtol=1e-6) and abs(r['var_total'] - vt) <= 1e-6 * vt
    assert r['n_solves'] == 64
    ctx.close()


def test_time_dilution_ragged():
    from paper_2607_05157_b300 import Context, trace_estimate, WD_HUTCH, WD_DIL_TIME
    dims = (2, 4, 6, 4)
    U = synth.gauge_field(dims, 0.5, 7)
    Dinv = solver.dense_inverse(wilson.sparse_matrix(U, 0.13, BC))
    ctx = Context(dims, U, 0.13, BC)
    r = trace_estimate(ctx.h, WD_HUTCH, 1 | WD_DIL_TIME, 5, dims[3], seed=9, op=1, prec=1, tol=1e-12, batch=7,
                       with_samples=True)
    ref = estimators.hutchinson(lambda v: Dinv @ v, dims, 9, 5, True, time_dilution=True)
    _close(r['samples'], ref)
    assert r['n_solves'] == 5 * dims[3]
    ctx.close()


@pytest.mark.parametrize("dims,d,dil", [((4, 4, 4, 4), 1, 12), ((4, 4, 4, 4), 2, 1), ((2, 4, 6, 4), 2, 12)])
def test_probing(dims, d, dil):
    from paper_2607_05157_b300 import Context, trace_estimate, WD_PROBE
    U = synth.gauge_field(dims, 0.5, 21)
    Dinv = solver.dense_inverse(wilson.sparse_matrix(U, 0.125, BC))
    ctx = Context(dims, U, 0.125, BC)
    nc, sigma = coloring.search(dims, d)
    col = coloring.colors(dims, sigma, nc)
    r = trace_estimate(ctx.h, WD_PROBE, dil, 3, dims[3], d=d, seed=77, op=1, prec=1, tol=1e-12, batch=50,
                       with_samples=True)
    ref = estimators.probing(lambda v: Dinv @ v, dims, 77, 3, True, col, nc, dil)
    _close(r['samples'], ref)
    assert r['n_solves'] == 3 * nc * dil
    ctx.close()


def _oracle_solve(U, kappa, shape):
    def f(v):
        x, it, res = solver.bicgstab(lambda y: wilson.apply(U, y.reshape(shape), kappa, BC), v, tol=1e-12)
        return x.reshape(-1)
    return f


def test_time_dilution_8x8x8x16_full_size():
    """The 8^3 x 16 workload in the benchmark's configuration (kappa 0.125,
    spread 0.5, time dilution, gamma5, mixed FP32 batched); sample 0's 16
    timeslices recomputed by the oracle's own BiCGStab."""
    from paper_2607_05157_b300 import Context, trace_estimate, WD_HUTCH, WD_DIL_TIME
    dims = (8, 8, 8, 16)
    U = synth.gauge_field(dims, 0.5, 1002)
    ctx = Context(dims, U, 0.125, BC)
    r = trace_estimate(ctx.h, WD_HUTCH, 1 | WD_DIL_TIME, 16, 16, seed=2002, op=1, prec=1, tol=1e-12,
                       with_samples=True)
    shape = synth.spinors(dims, 1, 0).shape[1:]
    solve = _oracle_solve(U, 0.125, shape)
    from oracle import noise
    eta = noise.rademacher(2002, 0, 12 * int(np.prod(dims)))
    ts = wilson.timeslice_of_dof(dims)
    scale = np.abs(r['samples'][0]).sum()
    for t in (0, 7, 15):                       # sampled outputs X_0(t)
        v = np.where(ts == t, eta, 0).astype(complex)
        ref = estimators.contract(v, solve(v), dims, True)[t]
        assert abs(r['samples'][0, t] - ref) <= 1e-8 * max(abs(ref), scale)
    ctx.close()


def test_probing_16x16x16x32_full_size():
    """The 16^3 x 32 lattice (kappa 0.13): probing d = 1 (2 colours), one
    sample, checked against the oracle's BiCGStab."""
    from paper_2607_05157_b300 import Context, trace_estimate, WD_PROBE
    dims = (16, 16, 16, 32)
    U = synth.gauge_field(dims, 0.5, 1003)
    ctx = Context(dims, U, 0.13, BC)
    r = trace_estimate(ctx.h, WD_PROBE, 1, 1, 32, d=1, seed=2003, op=1, prec=2, tol=1e-12, with_samples=True)
    nc, sigma = coloring.search(dims, 1)
    col = coloring.colors(dims, sigma, nc)
    shape = synth.spinors(dims, 1, 0).shape[1:]
    ref = estimators.probing(_oracle_solve(U, 0.13, shape), dims, 2003, 1, True, col, nc, 1)
    _close(r['samples'], ref)
    ctx.close()


def _diluted_reference(Dinv, dims, seed, N, gamma5, col, nc, dil):
    """X_i(t) of time dilution combined with colour x spin-colour dilution,
    composed from the oracle's noise, masks and contraction: the RHS of
    sample i are eta_i masked to (colour, component, timeslice t0)."""
    from oracle import noise
    n = 12 * int(np.prod(dims))
    ts = wilson.timeslice_of_dof(dims)
    masks = estimators.probing_masks(col, nc, dil)
    out = np.zeros((N, dims[3]), np.complex128)
    for i in range(N):
        eta = noise.rademacher(seed, i, n)
        for m in masks:
            for t0 in range(dims[3]):
                v = np.where(m & (ts == t0), eta, 0).astype(complex)
                out[i] += estimators.contract(v, Dinv @ v, dims, gamma5)
    return out


@pytest.mark.parametrize("dims,method,d,dil,op", [
    ((2, 4, 4, 2), 0, 0, 1, 1),      # T = 2: the Schur source reaches both timeslices
    ((4, 4, 4, 4), 1, 1, 12, 1),     # probing x spin-colour x time dilution, gamma5
    ((2, 4, 6, 4), 1, 2, 1, 0),      # B = 1: the full contraction with the odd solution
    ((4, 2, 2, 6), 0, 0, 12, 1),     # Hutchinson x spin-colour x time dilution
])
def test_time_diluted_variants(dims, method, d, dil, op):
    """Time dilution in every combination the estimator supports. With
    B = gamma5 the contraction uses the Schur source and the even solution
    only (X(t0) = bhat^dag g5 x_e + eta_o^dag g5 eta_o); the Schur-source
    stencil skips timeslices the source cannot reach. Per-sample values
    against the oracle's dense inverse."""
    from paper_2607_05157_b300 import Context, trace_estimate, WD_DIL_TIME
    U = synth.gauge_field(dims, 0.5, 31)
    Dinv = solver.dense_inverse(wilson.sparse_matrix(U, 0.125, BC))
    if method == 1:
        nc, sigma = coloring.search(dims, d)
        col = coloring.colors(dims, sigma, nc)
    else:
        nc, col = 1, np.zeros(int(np.prod(dims)), np.int64)
    ctx = Context(dims, U, 0.125, BC)
    r = trace_estimate(ctx.h, method, dil | WD_DIL_TIME, 2, dims[3], d=d, seed=55, op=op, prec=1, tol=1e-12,
                       batch=13, with_samples=True)
    ref = _diluted_reference(Dinv, dims, 55, 2, bool(op), col, nc, dil)
    _close(r['samples'], ref)
    assert r['n_solves'] == 2 * nc * dil * dims[3]
    ctx.close()


@pytest.mark.parametrize("dims,d,dil,op", [((4, 4, 4, 4), 2, 1, 1), ((4, 2, 6, 4), 1, 12, 0)])
def test_probing_3d_timeslice_colouring(dims, d, dil, op):
    """Probing with the colouring of one timeslice (Eq. 15 with n_D = 3,
    WD_COLOR_3D) under time dilution: every timeslice is coloured alike and
    probed on its own; per-sample values against the oracle."""
    from paper_2607_05157_b300 import Context, trace_estimate, WD_PROBE, WD_DIL_TIME, WD_COLOR_3D
    U = synth.gauge_field(dims, 0.5, 32)
    Dinv = solver.dense_inverse(wilson.sparse_matrix(U, 0.125, BC))
    nc, sigma = coloring.search(dims[:3], d)
    col = np.tile(coloring.colors(dims[:3], sigma, nc), dims[3])
    ctx = Context(dims, U, 0.125, BC)
    r = trace_estimate(ctx.h, WD_PROBE, dil | WD_DIL_TIME | WD_COLOR_3D, 2, dims[3], d=d, seed=56, op=op, prec=1,
                       tol=1e-12, batch=29, with_samples=True)
    ref = _diluted_reference(Dinv, dims, 56, 2, bool(op), col, nc, dil)
    _close(r['samples'], ref)
    assert r['n_solves'] == 2 * nc * dil * dims[3]
    with pytest.raises(Exception):
        trace_estimate(ctx.h, WD_PROBE, dil | WD_COLOR_3D, 2, dims[3], d=d, seed=56, op=op, prec=1, tol=1e-12)
    ctx.close()
