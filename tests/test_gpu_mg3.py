"""Parity of the third multigrid level (Sec. 2 with L = 3) with the oracle:
P_2 built on the GPU from the same level-2 test vectors (restriction and
prolongation), the Galerkin operator D_3 = P_2^dag D_c P_2 applied to random
level-3 vectors (level-3 extents 1 and 2 make neighbours coincide), and the
three-level MLMC estimator per sample."""
import numpy as np
import pytest

import synth
from oracle import estimators, multigrid, solver, wilson
from tests.gpu_util import rel, to_dev

pytestmark = pytest.mark.gpu
BC = (1, 1, 1, -1)
CASES = [((4, 4, 4, 4), (2, 2, 2, 2), (2, 2, 2, 2)),
         ((4, 4, 4, 4), (2, 2, 2, 2), (1, 1, 2, 2)),
         ((4, 4, 4, 8), (2, 2, 2, 2), (2, 1, 1, 2)),
         ((4, 2, 6, 4), (2, 2, 3, 2), (1, 1, 1, 2))]


def _setup(dims, agg, agg2, kappa=0.12, nv=6, nv2=6, seed=1040):
    from paper_2607_05157_b300 import Context, wd_mg_setup, wd_mg3_setup
    U = synth.gauge_field(dims, 0.4, seed)
    tv = synth.test_vectors(dims, nv, 81)
    ctx = Context(dims, U, kappa, BC)
    wd_mg_setup(ctx.h, tv, nv, agg)
    D = wilson.sparse_matrix(U, kappa, BC)
    P1 = multigrid.prolongator(tv, dims, agg)
    D2 = multigrid.coarse_operator(D, P1)
    cd = multigrid.coarse_dims(dims, agg)
    rng = np.random.default_rng(83)
    tv2 = rng.standard_normal((nv2, D2.shape[0])) + 1j * rng.standard_normal((nv2, D2.shape[0]))
    wd_mg3_setup(ctx.h, tv2, nv2, agg2)
    P2 = multigrid.prolongator_coarse(tv2, cd, agg2, nv)
    D3 = multigrid.coarse_operator(D2, P2)
    return ctx, D, P1, D2, P2, D3


@pytest.mark.parametrize("dims,agg,agg2", CASES)
def test_transfer_and_level3_operator(dims, agg, agg2):
    import torch
    from paper_2607_05157_b300 import wd_restrict2, wd_prolong2, wd_coarse3_apply
    ctx, D, P1, D2, P2, D3 = _setup(dims, agg, agg2)
    n2, n3 = P2.shape
    Vc, Vcc = n2 // 12, n3 // 12
    rng = np.random.default_rng(5)
    y2 = rng.standard_normal((3, n2)) + 1j * rng.standard_normal((3, n2))
    y3 = rng.standard_normal((3, n3)) + 1j * rng.standard_normal((3, n3))
    r = wd_restrict2(ctx.h, to_dev(y2.reshape(3, Vc, 12)),
                     torch.empty((3, Vcc, 12), dtype=torch.complex128, device='cuda')).cpu().numpy().reshape(3, -1)
    p = wd_prolong2(ctx.h, to_dev(y3.reshape(3, Vcc, 12)),
                    torch.empty((3, Vc, 12), dtype=torch.complex128, device='cuda')).cpu().numpy().reshape(3, -1)
    a = wd_coarse3_apply(ctx.h, to_dev(y3.reshape(3, Vcc, 12)),
                         torch.empty((3, Vcc, 12), dtype=torch.complex128, device='cuda')).cpu().numpy().reshape(3, -1)
    for i in range(3):
        assert rel(r[i], P2.conj().T @ y2[i]) < 1e-13
        assert rel(p[i], P2 @ y3[i]) < 1e-13
        assert rel(a[i], D3 @ y3[i]) < 1e-12
    ctx.close()


@pytest.mark.parametrize("gamma5,prec", [(1, 1), (0, 0)])
def test_mlmc3_per_sample(gamma5, prec):
    from paper_2607_05157_b300 import trace_estimate_mlmc3
    dims, agg, agg2 = (4, 4, 4, 4), (2, 2, 2, 2), (1, 1, 2, 2)
    ctx, D, P1, D2, P2, D3 = _setup(dims, agg, agg2)
    N1, N2, N3 = 3, 4, 5
    r = trace_estimate_mlmc3(ctx.h, N1, N2, N3, dims[3], seed=2030, op=gamma5, prec=prec, tol=1e-12, batch=2)
    Dinv = solver.dense_inverse(D)
    D2inv = solver.dense_inverse(D2)
    D3inv = solver.dense_inverse(D3)
    R = estimators.mlmc3(lambda v: Dinv @ v, lambda v: D2inv @ v, lambda v: D3inv @ v, P1, P2, dims, 2030,
                         N1, N2, N3, bool(gamma5))
    for l in range(3):
        got, ref = r['samples%d' % (l + 1)], R[l]
        scale = max(np.abs(ref).max(), np.abs(ref).sum(1).mean())
        assert np.abs(got - ref).max() <= 1e-8 * scale, (l, np.abs(got - ref).max() / scale)
    tots = [estimators.mean_and_variance(R[l]) for l in range(3)]
    total = sum(t[2] for t in tots)
    vtot = sum(t[3] / n for t, n in zip(tots, (N1, N2, N3)))
    assert abs(r['total'] - total) <= 1e-8 * sum(np.abs(R[l]).sum(1).mean() for l in range(3))
    assert abs(r['var_total'] - vtot) <= 1e-6 * vtot
    assert r['n_solves'] == 2 * N1 + 2 * N2 + N3
    ctx.close()


def test_gpu_level2_test_vectors_give_orthonormal_p2():
    """Level-2 test vectors from inverse iterations on the GPU (no host
    input): P_2^dag P_2 = I, seen as restrict2(prolong2(y)) = y."""
    import torch
    from paper_2607_05157_b300 import Context, wd_mg_setup, wd_mg3_setup, wd_restrict2, wd_prolong2
    dims = (8, 8, 8, 8)
    ctx = Context(dims, synth.gauge_field(dims, 0.5, 3), 0.13, BC)
    wd_mg_setup(ctx.h, None, 24, (2, 2, 2, 2), tv_iters=2, seed=11)
    wd_mg3_setup(ctx.h, None, 12, (2, 2, 2, 2), tv_iters=2, seed=12)
    Vcc, n3 = 16, 24
    rng = np.random.default_rng(2)
    y = rng.standard_normal((2, Vcc, n3)) + 1j * rng.standard_normal((2, Vcc, n3))
    f = wd_prolong2(ctx.h, to_dev(y), torch.empty((2, 256, 48), dtype=torch.complex128, device='cuda'))
    back = wd_restrict2(ctx.h, f, torch.empty((2, Vcc, n3), dtype=torch.complex128, device='cuda')).cpu().numpy()
    assert rel(back, y) < 1e-13
    ctx.close()
