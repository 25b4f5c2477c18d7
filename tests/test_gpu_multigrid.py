"""Parity of the two-level hierarchy (row a8) with the oracle: the prolongator
built on the GPU from the same test vectors, restriction and prolongation,
the Galerkin coarse operator D_c = P^dag D P (Eq. 7) applied to random coarse
vectors, coarse solves, and the two-level MLMC estimator (Eqs. 9-12) per sample.
Lattices include coarse extents 1 and 2 (neighbours coincide) and a ragged one."""
import numpy as np
import pytest

import synth
from oracle import estimators, multigrid, solver, wilson
from tests.gpu_util import rel, to_dev

pytestmark = pytest.mark.gpu
BC = (1, 1, 1, -1)
CASES = [((4, 4, 4, 4), (2, 2, 2, 2), 6), ((4, 4, 4, 4), (4, 4, 4, 4), 12), ((4, 2, 6, 4), (2, 2, 3, 2), 6),
         ((8, 8, 8, 8), (4, 4, 4, 4), 24)]


def _setup(dims, agg, nv, kappa=0.13, seed=1004):
    from paper_2607_05157_b300 import Context, wd_mg_setup
    U = synth.gauge_field(dims, 0.5, seed)
    tv = synth.test_vectors(dims, nv, 77)
    ctx = Context(dims, U, kappa, BC)
    wd_mg_setup(ctx.h, tv, nv, agg)
    D = wilson.sparse_matrix(U, kappa, BC)
    P = multigrid.prolongator(tv, dims, agg)
    return ctx, U, D, P


def _coarse_shape(dims, agg, nv, nrhs):
    Vc = int(np.prod([L // a for L, a in zip(dims, agg)]))
    return (nrhs, Vc, 2 * nv)


@pytest.mark.parametrize("dims,agg,nv", CASES)
def test_transfer_and_coarse_operator(dims, agg, nv):
    from paper_2607_05157_b300 import wd_restrict, wd_prolong, wd_coarse_apply
    import torch
    ctx, U, D, P = _setup(dims, agg, nv)
    Dc = multigrid.coarse_operator(D, P)
    rng = np.random.default_rng(5)
    cs = _coarse_shape(dims, agg, nv, 3)
    yc = rng.standard_normal(cs) + 1j * rng.standard_normal(cs)
    v = synth.spinors(dims, 3, 6)
    # restriction P^dag v and prolongation P y
    rc = wd_restrict(ctx.h, to_dev(v), torch.empty(cs, dtype=torch.complex128, device='cuda')).cpu().numpy()
    pf = wd_prolong(ctx.h, to_dev(yc), torch.empty(v.shape, dtype=torch.complex128, device='cuda')).cpu().numpy()
    for r in range(3):
        assert rel(rc[r].reshape(-1), P.conj().T @ v[r].reshape(-1)) < 1e-12
        assert rel(pf[r].reshape(-1), P @ yc[r].reshape(-1)) < 1e-12
    # coarse operator, FP64 and mixed (BF16 tensor-core or FP32 operands)
    y64 = wd_coarse_apply(ctx.h, to_dev(yc), torch.empty(cs, dtype=torch.complex128, device='cuda'), 0).cpu().numpy()
    ylo = wd_coarse_apply(ctx.h, to_dev(yc), torch.empty(cs, dtype=torch.complex128, device='cuda'), 1).cpu().numpy()
    for r in range(3):
        ref = Dc @ yc[r].reshape(-1)
        assert rel(y64[r].reshape(-1), ref) < 1e-12
        assert rel(ylo[r].reshape(-1), ref) < 2e-2
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_coarse_solve(prec):
    from paper_2607_05157_b300 import wd_coarse_solve
    import torch
    dims, agg, nv = (4, 4, 4, 4), (2, 2, 2, 2), 6
    ctx, U, D, P = _setup(dims, agg, nv)
    Dc = multigrid.coarse_operator(D, P).toarray()
    cs = _coarse_shape(dims, agg, nv, 2)
    rng = np.random.default_rng(9)
    b = rng.standard_normal(cs) + 1j * rng.standard_normal(cs)
    x = torch.empty(cs, dtype=torch.complex128, device='cuda')
    res = wd_coarse_solve(ctx.h, to_dev(b), x, 1e-10, prec)
    x = x.cpu().numpy()
    for r in range(2):
        tr = np.linalg.norm(b[r].reshape(-1) - Dc @ x[r].reshape(-1)) / np.linalg.norm(b[r])
        assert tr <= 1e-10 * 1.01 and abs(tr - res[r]) < 1e-11
    ctx.close()


@pytest.mark.parametrize("gamma5", [0, 1])
def test_mlmc2_per_sample(gamma5):
    from paper_2607_05157_b300 import trace_estimate, wd_mlmc_level2_samples, WD_MLMC2
    dims, agg, nv = (4, 4, 4, 4), (2, 2, 2, 2), 6
    ctx, U, D, P = _setup(dims, agg, nv, kappa=0.12, seed=1001)
    N1, N2 = 6, 10
    r = trace_estimate(ctx.h, WD_MLMC2, 1, N1, dims[3], n2=N2, seed=2004, op=gamma5, prec=1, tol=1e-12,
                       with_samples=True)
    X2 = wd_mlmc_level2_samples(ctx.h, N2, dims[3])
    Dinv = solver.dense_inverse(D)
    Dcinv = solver.dense_inverse(multigrid.coarse_operator(D, P))
    R1, R2 = estimators.mlmc2(lambda v: Dinv @ v, lambda v: Dcinv @ v, P, dims, 2004, N1, N2, bool(gamma5))
    for got, ref in ((r['samples'], R1), (X2, R2)):
        scale = max(np.abs(ref).max(), np.abs(ref).sum(1).mean())
        assert np.abs(got - ref).max() <= 1e-8 * scale
    m1, v1, mt1, vt1 = estimators.mean_and_variance(R1)
    m2, v2, mt2, vt2 = estimators.mean_and_variance(R2)
    assert abs(r['total'] - (mt1 + mt2)) <= 1e-8 * (np.abs(R1).sum(1).mean() + np.abs(R2).sum(1).mean())
    assert abs(r['var_total'] - (vt1 / N1 + vt2 / N2)) <= 1e-6 * (vt1 / N1 + vt2 / N2)
    assert r['n_solves'] == 2 * N1 + N2
    ctx.close()


@pytest.mark.parametrize("gamma5,dil,time_dil,d", [(1, 12, False, 1), (0, 1, False, 2), (1, 1, True, 1)])
def test_mlmc2_probe_per_sample(gamma5, dil, time_dil, d):
    """Two-level MLMC with probing on level 1 (the combination of the
    paper's outlook): per-sample level-1 values (probing x dilution [x time]
    vectors, fine minus coarse-corrected solves) and level-2 values against
    the oracle with the same prolongator, element by element."""
    from paper_2607_05157_b300 import trace_estimate, wd_mlmc_level2_samples, WD_MLMC2_PROBE, WD_DIL_TIME
    from oracle import coloring
    dims, agg, nv = (4, 4, 4, 4), (2, 2, 2, 2), 6
    ctx, U, D, P = _setup(dims, agg, nv, kappa=0.12, seed=1001)
    nc, sigma = coloring.search(dims, d)
    col = coloring.colors(dims, sigma, nc)
    N1, N2 = 2, 6
    flags = dil | (WD_DIL_TIME if time_dil else 0)
    r = trace_estimate(ctx.h, WD_MLMC2_PROBE, flags, N1, dims[3], n2=N2, d=d, seed=2014, op=gamma5, prec=1,
                       tol=1e-12, batch=37, with_samples=True)
    X2 = wd_mlmc_level2_samples(ctx.h, N2, dims[3])
    Dinv = solver.dense_inverse(D)
    Dcinv = solver.dense_inverse(multigrid.coarse_operator(D, P))
    R1, R2 = estimators.mlmc2_probe(lambda v: Dinv @ v, lambda v: Dcinv @ v, P, dims, 2014, N1, N2, bool(gamma5),
                                    col, nc, dil, time_dil)
    for got, ref in ((r['samples'], R1), (X2, R2)):
        scale = max(np.abs(ref).max(), np.abs(ref).sum(1).mean())
        assert np.abs(got - ref).max() <= 1e-8 * scale
    m1, v1, mt1, vt1 = estimators.mean_and_variance(R1)
    m2, v2, mt2, vt2 = estimators.mean_and_variance(R2)
    assert abs(r['total'] - (mt1 + mt2)) <= 1e-8 * (np.abs(R1).sum(1).mean() + np.abs(R2).sum(1).mean())
    m = nc * dil * (dims[3] if time_dil else 1)
    assert r['n_solves'] == 2 * N1 * m + N2
    ctx.close()


@pytest.mark.parametrize("dims,agg,nv,d2,cfull", [((4, 4, 4, 4), (2, 2, 2, 2), 6, 1, True),
                                                 ((4, 4, 4, 4), (2, 2, 2, 2), 6, 0, False),
                                                 ((4, 2, 6, 4), (2, 2, 3, 2), 6, 2, True)])
def test_mlmc_probe_both_levels_per_sample(dims, agg, nv, d2, cfull):
    """Probing on both levels: level 1 with the fine probing vectors, level 2
    with the colouring of the coarse torus x coarse-dof dilution; per-sample
    values of both levels against the oracle."""
    from paper_2607_05157_b300 import trace_estimate_mlmc_probe
    from oracle import coloring
    ctx, U, D, P = _setup(dims, agg, nv, kappa=0.12, seed=1001)
    nc, sigma = coloring.search(dims, 1)
    col = coloring.colors(dims, sigma, nc)
    cd = multigrid.coarse_dims(dims, agg)
    if d2 > 0:
        nc2, sig2 = coloring.search(cd, d2)
        ccol = coloring.colors(cd, sig2, nc2)
    else:
        nc2, ccol = 1, np.zeros(int(np.prod(cd)), np.int64)
    cdil = 2 * nv if cfull else 1
    N1, N2 = 2, 3
    r = trace_estimate_mlmc_probe(ctx.h, 12, 1, N1, cdil, d2, N2, dims[3], seed=2016, op=1, prec=1, tol=1e-12,
                                  batch=29)
    Dinv = solver.dense_inverse(D)
    Dcinv = solver.dense_inverse(multigrid.coarse_operator(D, P))
    R1, R2 = estimators.mlmc2_probe(lambda v: Dinv @ v, lambda v: Dcinv @ v, P, dims, 2016, N1, N2, True, col, nc,
                                    12, coarse_col=ccol, coarse_nc=nc2, coarse_dil=cdil)
    for got, ref in ((r['samples1'], R1), (r['samples2'], R2)):
        scale = max(np.abs(ref).max(), np.abs(ref).sum(1).mean())
        assert np.abs(got - ref).max() <= 1e-8 * scale
    m1, v1, mt1, vt1 = estimators.mean_and_variance(R1)
    m2, v2, mt2, vt2 = estimators.mean_and_variance(R2)
    assert abs(r['total'] - (mt1 + mt2)) <= 1e-8 * (np.abs(R1).sum(1).mean() + np.abs(R2).sum(1).mean())
    assert abs(r['var_total'] - (vt1 / N1 + vt2 / N2)) <= 1e-6 * (vt1 / N1 + vt2 / N2)
    assert r['n_solves'] == 2 * N1 * nc * 12 + N2 * nc2 * cdil
    ctx.close()


def test_gpu_test_vectors_give_orthonormal_prolongator():
    """Test vectors from inverse iterations on the GPU (no host input):
    P^dag P = I holds, seen as restrict(prolong(y)) = y."""
    from paper_2607_05157_b300 import Context, wd_mg_setup, wd_restrict, wd_prolong
    import torch
    dims, agg, nv = (8, 8, 8, 8), (4, 4, 4, 4), 24
    ctx = Context(dims, synth.gauge_field(dims, 0.5, 3), 0.13, BC)
    wd_mg_setup(ctx.h, None, nv, agg, tv_iters=3, seed=11)
    cs = _coarse_shape(dims, agg, nv, 2)
    rng = np.random.default_rng(1)
    y = rng.standard_normal(cs) + 1j * rng.standard_normal(cs)
    f = wd_prolong(ctx.h, to_dev(y), torch.empty(ctx.field_shape(2), dtype=torch.complex128, device='cuda'))
    back = wd_restrict(ctx.h, f, torch.empty(cs, dtype=torch.complex128, device='cuda')).cpu().numpy()
    assert rel(back, y) < 1e-13
    ctx.close()


def test_tensor_core_coarse_stencil_16x16x16x32():
    """tcgen05 coarse stencil (BF16 operands, FP32 accumulate) on the 16^3 x 32
    lattice with 4^4 aggregates and 24 test vectors (48 x 48 blocks, 512 coarse
    sites), 130 right-hand sides (a full and a ragged 128-row tile).  Sampled
    RHS are checked against the oracle's P^dag D P x computed as restriction of
    the fine stencil applied to the prolonged vector."""
    import torch
    from paper_2607_05157_b300 import Context, wd_mg_setup, wd_coarse_apply
    dims, agg, nv = (16, 16, 16, 32), (4, 4, 4, 4), 24
    U = synth.gauge_field(dims, 0.5, 1003)
    tv = synth.test_vectors(dims, nv, 78)
    ctx = Context(dims, U, 0.13, BC)
    wd_mg_setup(ctx.h, tv, nv, agg)
    cs = _coarse_shape(dims, agg, nv, 130)
    rng = np.random.default_rng(12)
    x = rng.standard_normal(cs) + 1j * rng.standard_normal(cs)
    y = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 1).cpu().numpy()
    P = multigrid.prolongator(tv, dims, agg)
    shape = synth.spinors(dims, 1, 0).shape[1:]
    for r in (0, 127, 129):
        f = (P @ x[r].reshape(-1)).reshape(shape)
        ref = P.conj().T @ wilson.apply(U, f, 0.13, BC).reshape(-1)
        err = rel(y[r].reshape(-1), ref)
        # BF16 operands leave a ~1e-3 error floor: proves the tensor-core path ran
        # (the FP32 CUDA-core fallback would sit near 1e-7)
        assert 1e-5 < err < 2e-2, err
    ctx.close()
