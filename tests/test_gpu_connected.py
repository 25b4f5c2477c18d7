"""Parity of the connected pseudoscalar correlator with the two-level
multigrid decomposition (Sec. 4, Eqs. 16-20, L = 2; wd_connected_mlmc) with
the oracle on identical seeded noise: per-sample values of the (1,1), (1,2),
(2,1) and (2,2) terms, their means and variances, element by element."""
import numpy as np
import pytest

import synth
from oracle import connected, multigrid, solver, wilson

pytestmark = pytest.mark.gpu
BC = (1, 1, 1, -1)


def _setup(dims, agg, nv, kappa, seed):
    from paper_2607_05157_b300 import Context, wd_mg_setup
    U = synth.gauge_field(dims, 0.5, seed)
    tv = synth.test_vectors(dims, nv, 79)
    ctx = Context(dims, U, kappa, BC)
    wd_mg_setup(ctx.h, tv, nv, agg)
    D = wilson.sparse_matrix(U, kappa, BC)
    P = multigrid.prolongator(tv, dims, agg)
    return ctx, D, P


@pytest.mark.parametrize("dims,agg,nv,prec,batch", [((4, 4, 4, 4), (2, 2, 2, 2), 6, 1, 7),
                                                    ((4, 2, 6, 4), (2, 2, 3, 2), 6, 0, 0),
                                                    ((4, 4, 4, 4), (2, 2, 2, 2), 6, 2, 16)])
def test_connected_mlmc_per_sample(dims, agg, nv, prec, batch):
    from paper_2607_05157_b300 import wd_connected_mlmc
    ctx, D, P = _setup(dims, agg, nv, 0.12, 1021)
    T = dims[3]
    N1, N2 = 2, 5
    r = wd_connected_mlmc(ctx.h, N1, N2, T, seed=31, prec=prec, tol=1e-12, batch=batch, with_samples=True)
    Dinv = solver.dense_inverse(D)
    Dcinv = solver.dense_inverse(multigrid.coarse_operator(D, P))
    S1, S2 = connected.samples(lambda v: Dinv @ v, lambda v: Dcinv @ v, P, dims, 31, N1, N2)
    for got, ref in ((r['samples1'], S1), (r['samples2'], S2)):
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-8 * scale, np.abs(got - ref).max() / scale
    G, var = connected.estimate(S1, S2)
    assert np.abs(r['G'] - G).max() <= 1e-8 * np.abs(G).max()
    assert np.allclose(r['var'], var, rtol=1e-6, atol=1e-14 * np.abs(var).max())
    assert r['n_solves'] == 2 * N1 * T + N2 * T
    ctx.close()


def test_connected_total_tracks_exact_correlator():
    """The total of the estimate lies within 5 standard errors of the exact
    G(t) of Eq. 16 (dense inverse), and (1,2), (2,1) are conjugate."""
    from paper_2607_05157_b300 import wd_connected_mlmc
    dims, agg, nv = (4, 4, 4, 4), (2, 2, 2, 2), 6
    ctx, D, P = _setup(dims, agg, nv, 0.12, 1022)
    r = wd_connected_mlmc(ctx.h, 8, 32, dims[3], seed=5, prec=1, tol=1e-10)
    Dinv = solver.dense_inverse(D)
    G = connected.correlator_exact(Dinv, Dinv, dims)
    assert np.all(np.abs(r['G'][4] - G) <= 5 * np.sqrt(r['var'][4]) + 1e-10 * np.abs(G).max())
    assert np.abs(r['G'][2] - r['G'][1].conj()).max() <= 1e-12 * np.abs(r['G']).max()
    ctx.close()
