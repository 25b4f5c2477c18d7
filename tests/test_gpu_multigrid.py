"""Parity of the two-level hierarchy with the oracle: the prolongator
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


# Element-wise bound factor of the tensor-core coarse stencil against the FP64
# operator, per output component: BF16 operands (blocks and input rounded to
# nearest, unit roundoff u = 2^-8 each; the input first rounded to FP32), so
# 2u + u^2 + 2^-24 <= 2^-7 + 2^-15 per real product; |Re a Re x| + |Im a Im x|
# <= |a| |x| per complex product; FP32 accumulation of the 9 x 2 x 48 = 864
# real products of one component, gamma_n taken twice (1728 * 2^-24) for an
# accumulation order that is not IEEE pairwise:
#   |y - ref| <= U_TC * sum_b |A_b| |x|.
U_TC = 2.0 ** -7 + 2.0 ** -15 + 1728 * 2.0 ** -24
# The same with BF16-pair operands (WD_MIXED_FP32: v = hi + lo, lo the BF16
# rounding of v - hi, so |v - hi - lo| <= u^2 |v| = 2^-16 |v|): hi hi + lo hi +
# hi lo misses lo lo and the two representation errors, 3 * 2^-16 + 2^-24 <=
# 2^-14 per product, and accumulates 3 x 864 products (5184 * 2^-24 taken
# twice).  A dropped remainder product would leave a normwise error near
# 2^-9, far above the normwise limit REL_SPLIT.
U_SPLIT = 2.0 ** -14 + 5184 * 2.0 ** -24
REL_SPLIT = 5e-5


def u_tc(ncd):
    """U_TC for blocks of ncd coarse dofs: 18 ncd real products per output
    component (864 at ncd = 48, where it equals U_TC)."""
    return 2.0 ** -7 + 2.0 ** -15 + 2 * 18 * ncd * 2.0 ** -24


def u_split(ncd):
    """U_SPLIT for blocks of ncd coarse dofs (3 x 18 ncd products)."""
    return 2.0 ** -14 + 2 * 3 * 18 * ncd * 2.0 ** -24


def _coarse_nbr(cd):
    """Neighbour table of the coarse torus, lexicographic (x fastest):
    [Vc][9] with 0 the site, 1 + mu the forward and 5 + mu the backward one."""
    Vc = int(np.prod(cd))
    X = np.arange(Vc)
    c = [X % cd[0], (X // cd[0]) % cd[1], (X // (cd[0] * cd[1])) % cd[2], X // (cd[0] * cd[1] * cd[2])]
    def lexi(q):
        return q[0] + cd[0] * (q[1] + cd[1] * (q[2] + cd[2] * q[3]))
    nbr = np.empty((Vc, 9), np.int64)
    nbr[:, 0] = X
    for mu in range(4):
        for k, step in ((1 + mu, 1), (5 + mu, -1)):
            q = list(c)
            q[mu] = (q[mu] + step) % cd[mu]
            nbr[:, k] = lexi(q)
    return nbr


def _coarse_blocks(ctx, cd, ncd):
    """The 9 blocks A_b(X) of D_c, read off the GPU's FP64 coarse operator
    (held to the oracle's P^dag D P at 1e-12 by test_transfer_and_coarse_operator)
    by probing: a distance-2 colouring of the coarse torus (every extent >= 3,
    so that X and its 8 neighbours are 9 distinct sites with 9 distinct
    colours) and, per colour and coarse dof k, one application to the vector
    that is e_k on every site of that colour.  Returns (A [Vc][9][ncd][ncd], nbr)."""
    import torch
    from oracle import coloring
    from paper_2607_05157_b300 import wd_coarse_apply
    assert min(cd) >= 3
    nbr = _coarse_nbr(cd)
    Vc = nbr.shape[0]
    nc, sigma = coloring.search(cd, 2)
    col = coloring.colors(cd, sigma, nc)
    ncol = col[nbr]                                   # colours of the 9 sites each site couples to
    assert all(len(set(row)) == 9 for row in ncol)    # all distinct: each probe hits one block
    which = np.full((Vc, nc), -1, np.int64)           # block b of site Y that sees colour c (-1: none)
    for b in range(9):
        which[np.arange(Vc), ncol[:, b]] = b
    A = np.zeros((Vc, 9, ncd, ncd), np.complex128)
    probes = [(c, k) for c in range(nc) for k in range(ncd)]
    for i0 in range(0, len(probes), 128):
        chunk = probes[i0:i0 + 128]
        x = np.zeros((len(chunk), Vc, ncd), np.complex128)
        for r, (c, k) in enumerate(chunk):
            x[r, col == c, k] = 1.0
        y = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(x.shape, dtype=torch.complex128, device='cuda'),
                            0).cpu().numpy()
        for r, (c, k) in enumerate(chunk):
            hit = which[:, c] >= 0
            A[np.arange(Vc)[hit], which[hit, c], :, k] = y[r][hit]
            assert np.all(y[r][~hit] == 0)            # sites that see no probe get nothing
    return A, nbr


def _coarse_abs_bound(A, nbr, x):
    """sum_b |A_b(X)| |x(nbr_b(X))| for one coarse vector x [Vc][ncd]."""
    return sum(np.einsum('vij,vj->vi', np.abs(A[:, b]), np.abs(x[nbr[:, b]])) for b in range(9))


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
    # coarse operator, FP64 and mixed (tensor cores with BF16-pair or BF16
    # operands, or FP32 blocks), the mixed ones element by element against
    # U_SPLIT |D_c| |x| and U_TC |D_c| |x|
    y64 = wd_coarse_apply(ctx.h, to_dev(yc), torch.empty(cs, dtype=torch.complex128, device='cuda'), 0).cpu().numpy()
    ysp = wd_coarse_apply(ctx.h, to_dev(yc), torch.empty(cs, dtype=torch.complex128, device='cuda'), 1).cpu().numpy()
    ybf = wd_coarse_apply(ctx.h, to_dev(yc), torch.empty(cs, dtype=torch.complex128, device='cuda'), 2).cpu().numpy()
    Dabs = Dc.copy()
    Dabs.data = np.abs(Dabs.data)
    for r in range(3):
        ref = Dc @ yc[r].reshape(-1)
        assert rel(y64[r].reshape(-1), ref) < 1e-12
        assert rel(ysp[r].reshape(-1), ref) < REL_SPLIT
        assert rel(ybf[r].reshape(-1), ref) < 2e-2
        bound = Dabs @ np.abs(yc[r].reshape(-1))
        assert np.all(np.abs(ysp[r].reshape(-1) - ref) <= U_SPLIT * bound)
        assert np.all(np.abs(ybf[r].reshape(-1) - ref) <= U_TC * bound)
    ctx.close()


@pytest.mark.parametrize("case", [((4, 4, 4, 4), 2, 6), ((8, 8, 8, 8), 24, 6), ((4, 4, 4, 4), 40, 24),
                                  ((4, 4, 4, 4), 33, 48)])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_coarse_solve(prec, case):
    """True FP64 residual of the coarse solves against the oracle's D_c.  The
    mixed solves (prec 1, 2) take their residual by the recursive FP32 update
    r - D_c e once it is small; the reported residual still matches the true
    one to 1e-11 of |b|.  N_v = 24 and 48 give the double-float residual its
    48x48 and 96x96 blocks (the largest that fit its shared memory), with a
    ragged last tile of 32 RHS (40 = 32 + 8, 33 = 32 + 1)."""
    from paper_2607_05157_b300 import wd_coarse_solve
    import torch
    dims, nrhs, nv = case
    agg = (2, 2, 2, 2)
    ctx, U, D, P = _setup(dims, agg, nv)
    Dc = multigrid.coarse_operator(D, P).toarray()
    cs = _coarse_shape(dims, agg, nv, nrhs)
    rng = np.random.default_rng(9)
    b = rng.standard_normal(cs) + 1j * rng.standard_normal(cs)
    x = torch.empty(cs, dtype=torch.complex128, device='cuda')
    res = wd_coarse_solve(ctx.h, to_dev(b), x, 1e-10, prec)
    x = x.cpu().numpy()
    for r in range(nrhs):
        tr = np.linalg.norm(b[r].reshape(-1) - Dc @ x[r].reshape(-1)) / np.linalg.norm(b[r])
        assert tr <= 1e-10 * 1.01 and abs(tr - res[r]) < 1e-11, (r, tr, res[r])
    ctx.close()


@pytest.mark.parametrize("gamma5", [0, 1])
@pytest.mark.parametrize("N1", [6, 40, 70])
def test_mlmc2_per_sample(gamma5, N1):
    """Per-sample parity of both levels.  The level-1 restriction of the noise
    works on sign words of 64 samples in tiles of 16 samples per thread:
    N1 = 40 takes full tiles and a ragged one, N1 = 70 a full word and a
    second one of 6 samples."""
    from paper_2607_05157_b300 import trace_estimate, wd_mlmc_level2_samples, WD_MLMC2
    dims, agg, nv = (4, 4, 4, 4), (2, 2, 2, 2), 6
    ctx, U, D, P = _setup(dims, agg, nv, kappa=0.12, seed=1001)
    N2 = 10
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
    """tcgen05 coarse stencil (BF16 and BF16-pair operands, FP32 accumulate) on the 16^3 x 32
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
    y = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 2).cpu().numpy()
    ysp = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 1).cpu().numpy()
    y64 = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 0).cpu().numpy()
    P = multigrid.prolongator(tv, dims, agg)
    shape = synth.spinors(dims, 1, 0).shape[1:]
    A, nbr = _coarse_blocks(ctx, [L // a for L, a in zip(dims, agg)], 2 * nv)
    for r in (0, 127, 129):
        f = (P @ x[r].reshape(-1)).reshape(shape)
        ref = P.conj().T @ wilson.apply(U, f, 0.13, BC).reshape(-1)
        assert rel(y64[r].reshape(-1), ref) < 1e-12
        err = rel(y[r].reshape(-1), ref)
        # BF16 operands leave a ~1e-3 error floor: proves the tensor-core path ran
        # (the FP32 CUDA-core fallback would sit near 1e-7)
        assert 1e-5 < err < 2e-2, err
        assert rel(ysp[r].reshape(-1), ref) < REL_SPLIT
    # every element of every RHS against the probed blocks
    for r in range(x.shape[0]):
        bound = _coarse_abs_bound(A, nbr, x[r])
        assert np.all(np.abs(y[r] - y64[r]) <= U_TC * bound), r
        assert np.all(np.abs(ysp[r] - y64[r]) <= U_SPLIT * bound), r
    ctx.close()


def test_tensor_core_coarse_stencil_24x24x24x48_sampled():
    """The two-level workload's coarse lattice (24^3 x 48, 4^4 aggregates, 24
    test vectors: 2592 coarse sites of 48 x 48 blocks), 200 RHS (a full and a
    ragged 128-row tile): every element of sampled RHS against the FP64 coarse
    operator within U_TC |A| |x| (BF16) and U_SPLIT |A| |x| (BF16 pairs), the
    blocks probed from that operator."""
    import torch
    from paper_2607_05157_b300 import Context, wd_mg_setup, wd_coarse_apply
    dims, agg, nv = (24, 24, 24, 48), (4, 4, 4, 4), 24
    ctx = Context(dims, synth.gauge_field(dims, 0.5, 1004), 0.13, BC)
    wd_mg_setup(ctx.h, None, nv, agg, tv_iters=1, seed=5)
    cs = _coarse_shape(dims, agg, nv, 200)
    rng = np.random.default_rng(13)
    x = rng.standard_normal(cs) + 1j * rng.standard_normal(cs)
    y = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 2).cpu().numpy()
    ysp = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 1).cpu().numpy()
    y64 = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 0).cpu().numpy()
    A, nbr = _coarse_blocks(ctx, [L // a for L, a in zip(dims, agg)], 2 * nv)
    for r in (0, 1, 64, 127, 128, 199):
        bound = _coarse_abs_bound(A, nbr, x[r])
        assert np.all(np.abs(y[r] - y64[r]) <= U_TC * bound), r
        assert 1e-5 < rel(y[r], y64[r]) < 2e-2
        assert np.all(np.abs(ysp[r] - y64[r]) <= U_SPLIT * bound), r
        assert rel(ysp[r], y64[r]) < REL_SPLIT
    ctx.close()


@pytest.mark.parametrize("nrhs", [1, 9, 40, 64, 129, 257])
def test_tensor_core_coarse_stencil_rhs_counts(nrhs):
    """RHS counts at the edges of the tiling: one row, counts that are not a
    multiple of 8 (the input rows are padded to 8), a last tile of one RHS,
    three tiles; with BF16 pairs, tiles of at most 64 RHS stack their Re and
    Im rows into one MMA (40: the Im rows straddle two lane quarters, 64: they
    fill the upper two).  Every element against the FP64 coarse operator
    within U_TC (BF16) and U_SPLIT (BF16 pairs), on 12^4 with 4^4 aggregates."""
    import torch
    from paper_2607_05157_b300 import Context, wd_mg_setup, wd_coarse_apply
    dims, agg, nv = (12, 12, 12, 12), (4, 4, 4, 4), 24
    ctx = Context(dims, synth.gauge_field(dims, 0.5, 1007), 0.13, BC)
    wd_mg_setup(ctx.h, synth.test_vectors(dims, nv, 80), nv, agg)
    cs = _coarse_shape(dims, agg, nv, nrhs)
    rng = np.random.default_rng(15 + nrhs)
    x = rng.standard_normal(cs) + 1j * rng.standard_normal(cs)
    y = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 2).cpu().numpy()
    ysp = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 1).cpu().numpy()
    y64 = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 0).cpu().numpy()
    A, nbr = _coarse_blocks(ctx, [L // a for L, a in zip(dims, agg)], 2 * nv)
    for r in sorted({0, nrhs // 2, nrhs - 1, min(nrhs - 1, 128)}):
        bound = _coarse_abs_bound(A, nbr, x[r])
        assert np.all(np.abs(y[r] - y64[r]) <= U_TC * bound), r
        assert np.all(np.abs(ysp[r] - y64[r]) <= U_SPLIT * bound), r
        assert rel(ysp[r], y64[r]) < REL_SPLIT
    ctx.close()


def test_tensor_core_coarse_stencil_96_dofs():
    """The second shape of the tensor-core stencil: 48 test vectors (96 x 96
    blocks, MMA N = 192, one accumulator set of 512 TMEM columns) on 12^4 with
    4^4 aggregates (3^4 coarse sites), 70 RHS (one ragged tile): every element
    of every RHS against the FP64 coarse operator within u_tc / u_split (96),
    the blocks probed from that operator."""
    import torch
    from paper_2607_05157_b300 import Context, wd_mg_setup, wd_coarse_apply
    dims, agg, nv = (12, 12, 12, 12), (4, 4, 4, 4), 48
    ctx = Context(dims, synth.gauge_field(dims, 0.5, 1006), 0.13, BC)
    wd_mg_setup(ctx.h, synth.test_vectors(dims, nv, 79), nv, agg)
    cs = _coarse_shape(dims, agg, nv, 70)
    rng = np.random.default_rng(14)
    x = rng.standard_normal(cs) + 1j * rng.standard_normal(cs)
    y = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 2).cpu().numpy()
    ysp = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 1).cpu().numpy()
    y64 = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 0).cpu().numpy()
    A, nbr = _coarse_blocks(ctx, [L // a for L, a in zip(dims, agg)], 2 * nv)
    for r in range(x.shape[0]):
        bound = _coarse_abs_bound(A, nbr, x[r])
        assert np.all(np.abs(y[r] - y64[r]) <= u_tc(2 * nv) * bound), r
        assert np.all(np.abs(ysp[r] - y64[r]) <= u_split(2 * nv) * bound), r
        assert 1e-5 < rel(y[r], y64[r]) < 2e-2
        assert rel(ysp[r], y64[r]) < REL_SPLIT
    ctx.close()


def test_gpu_test_vectors_match_oracle_inverse_iteration():
    """wd_mg_test_vectors against the oracle's inverse iteration (Sec. 2's
    setup) from the same Rademacher starts, after 1, 2 and 3 iterations.  Each
    GPU solve stops at a relative residual eps = 1e-6 while the oracle solves to
    1e-12, so the normalised map v -> D^{-1} v / |D^{-1} v| (Lipschitz constant
    at most 2 cond(D)) bounds the error of iterate i by
    e_i <= 2 cond(D) (e_{i-1} + eps), e_0 = 0; cond(D) from the dense SVD."""
    import torch
    from paper_2607_05157_b300 import Context, wd_mg_test_vectors
    dims, kappa, nv, seed, eps = (4, 4, 4, 4), 0.12, 12, 31, 1e-6
    U = synth.gauge_field(dims, 0.5, 1004)
    ctx = Context(dims, U, kappa, BC)
    sv = np.linalg.svd(wilson.sparse_matrix(U, kappa, BC).toarray(), compute_uv=False)
    cond = sv[0] / sv[-1]
    e_prev = 0.0
    for iters in (1, 2, 3):
        out = torch.empty((nv,) + synth.spinors(dims, 1, 0).shape[1:], dtype=torch.complex128, device='cuda')
        got = wd_mg_test_vectors(ctx.h, nv, iters, seed, out).cpu().numpy()
        ref = multigrid.test_vectors(lambda v: wilson.apply(U, v, kappa, BC), dims, nv, iters, seed)
        e = max(np.linalg.norm((got[k] - ref[k]).reshape(-1)) for k in range(nv))
        bound = 2 * cond * (e_prev + eps)
        assert e <= bound, (iters, e, bound)
        assert all(abs(np.linalg.norm(got[k]) - 1.0) < 1e-12 for k in range(nv))
        e_prev = e
    ctx.close()


@pytest.mark.parametrize("dims,agg,nv", [((4, 4, 4, 4), (2, 2, 2, 2), 12), ((8, 8, 8, 8), (4, 4, 4, 4), 24)])
def test_gpu_built_prolongator_matches_oracle_mgs(dims, agg, nv):
    """wd_mg_setup(tv = NULL) builds P from its own test vectors: P^dag v and
    P y agree element by element with the oracle's prolongator (block MGS,
    Sec. 2) of the same GPU test vectors (wd_mg_test_vectors, same seed)."""
    import torch
    from paper_2607_05157_b300 import Context, wd_mg_setup, wd_mg_test_vectors, wd_restrict, wd_prolong
    U = synth.gauge_field(dims, 0.5, 1005)
    ctx = Context(dims, U, 0.13, BC)
    shape = synth.spinors(dims, 1, 0).shape[1:]
    tv = wd_mg_test_vectors(ctx.h, nv, 3, 9, torch.empty((nv,) + shape, dtype=torch.complex128,
                                                          device='cuda')).cpu().numpy()
    wd_mg_setup(ctx.h, None, nv, agg, tv_iters=3, seed=9)
    P = multigrid.prolongator(tv, dims, agg)
    v = synth.spinors(dims, 2, 21)
    cs = _coarse_shape(dims, agg, nv, 2)
    rng = np.random.default_rng(22)
    y = rng.standard_normal(cs) + 1j * rng.standard_normal(cs)
    rc = wd_restrict(ctx.h, to_dev(v), torch.empty(cs, dtype=torch.complex128, device='cuda')).cpu().numpy()
    pf = wd_prolong(ctx.h, to_dev(y), torch.empty(v.shape, dtype=torch.complex128, device='cuda')).cpu().numpy()
    for r in range(2):
        ref_r = P.conj().T @ v[r].reshape(-1)
        ref_p = P @ y[r].reshape(-1)
        assert np.abs(rc[r].reshape(-1) - ref_r).max() <= 1e-12 * np.abs(ref_r).max()
        assert np.abs(pf[r].reshape(-1) - ref_p).max() <= 1e-12 * np.abs(ref_p).max()
    ctx.close()


def test_tensor_core_bounded_wait_gives_up_and_context_stays_usable(monkeypatch):
    """The failure path of the tensor-core coarse stencil, without any fault:
    WD_TEST_TC_STALL=1 makes the MMA issuer wait, with a short limit, on a
    barrier nothing arrives on.  The kernel gives up, lets its TMA copies land,
    frees its TMEM and returns; wd_coarse_apply reports WD_ETIMEOUT, and the
    next call on the same context gives the normal result bit for bit."""
    import torch
    from paper_2607_05157_b300 import Context, WDError, wd_mg_setup, wd_coarse_apply
    from paper_2607_05157_b300._lib import WD_ETIMEOUT
    dims, agg, nv = (8, 8, 8, 8), (4, 4, 4, 4), 24
    ctx = Context(dims, synth.gauge_field(dims, 0.5, 1004), 0.13, BC)
    wd_mg_setup(ctx.h, synth.test_vectors(dims, nv, 77), nv, agg)
    cs = _coarse_shape(dims, agg, nv, 130)
    rng = np.random.default_rng(4)
    x = to_dev(rng.standard_normal(cs) + 1j * rng.standard_normal(cs))
    y0 = wd_coarse_apply(ctx.h, x, torch.empty(cs, dtype=torch.complex128, device='cuda'), 1).cpu().numpy()
    monkeypatch.setenv('WD_TEST_TC_STALL', '1')
    with pytest.raises(WDError) as e:
        wd_coarse_apply(ctx.h, x, torch.empty(cs, dtype=torch.complex128, device='cuda'), 1)
    assert e.value.status == WD_ETIMEOUT
    monkeypatch.delenv('WD_TEST_TC_STALL')
    y1 = wd_coarse_apply(ctx.h, x, torch.empty(cs, dtype=torch.complex128, device='cuda'), 1).cpu().numpy()
    assert np.array_equal(y0, y1)
    ctx.close()


def test_fp32_coarse_stencil_tiled(monkeypatch):
    """The FP32 coarse stencil on the CUDA cores (the recursive residual
    updates of the coarse solves): 40 RHS take the kernel tiled over 32 RHS
    (one full tile and a ragged one), 8 RHS the one-RHS-per-thread kernel.
    Element by element inside the FP32 bound of a 9 ncd-term dot product with
    rounded inputs, (2 + 9 ncd) 2^-24 sum |A||x|, and the two kernels give
    the same bits (the same products in the same order)."""
    import torch
    from paper_2607_05157_b300 import wd_coarse_apply
    monkeypatch.setenv('WD_COARSE_FP32', '1')
    dims, agg, nv = (6, 6, 6, 6), (2, 2, 2, 2), 6
    ctx, U, D, P = _setup(dims, agg, nv)
    ncd = 2 * nv
    Dc = multigrid.coarse_operator(D, P).toarray()
    nbr = _coarse_nbr(tuple(L // a for L, a in zip(dims, agg)))
    Vc = nbr.shape[0]
    A = np.empty((Vc, 9, ncd, ncd), np.complex128)      # the oracle's blocks
    for X in range(Vc):
        for b in range(9):
            A[X, b] = Dc[X * ncd:(X + 1) * ncd, nbr[X, b] * ncd:(nbr[X, b] + 1) * ncd]
    cs = _coarse_shape(dims, agg, nv, 40)
    rng = np.random.default_rng(21)
    x = rng.standard_normal(cs) + 1j * rng.standard_normal(cs)
    y = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 1).cpu().numpy()
    y8 = wd_coarse_apply(ctx.h, to_dev(x[:8]), torch.empty((8,) + cs[1:], dtype=torch.complex128, device='cuda'),
                         1).cpu().numpy()
    assert np.array_equal(y[:8], y8)
    u = (2 + 9 * ncd) * 2.0 ** -24
    for r in range(40):
        ref = (Dc @ x[r].reshape(-1)).reshape(Vc, ncd)
        assert np.all(np.abs(y[r] - ref) <= u * _coarse_abs_bound(A, nbr, x[r])), r
    ctx.close()


def test_setup_again_after_new_links():
    """The path of the end-to-end loop: wd_update_gauge (new links, new kappa)
    and a second wd_mg_setup of the same geometry on the same context, which
    overwrites the multigrid buffers in place.  The coarse operator is then
    the oracle's P^dag D P of the new links (FP64 to 1e-12, the tensor-core
    BF16-pair path element by element); a third setup of another N_v
    allocates afresh and is right as well."""
    import torch
    from paper_2607_05157_b300 import Context, wd_mg_setup, wd_coarse_apply, wd_update_gauge
    dims, agg = (8, 8, 8, 8), (2, 2, 2, 2)
    ctx = Context(dims, synth.gauge_field(dims, 0.5, 1010), 0.13, BC)
    wd_mg_setup(ctx.h, synth.test_vectors(dims, 24, 80), 24, agg)
    U2 = synth.gauge_field(dims, 0.5, 1011)
    wd_update_gauge(ctx.h, U2, 0.12)
    D2 = wilson.sparse_matrix(U2, 0.12, BC)
    rng = np.random.default_rng(17)
    for nv, seed in ((24, 81), (12, 82)):
        tv = synth.test_vectors(dims, nv, seed)
        wd_mg_setup(ctx.h, tv, nv, agg)
        Dc = multigrid.coarse_operator(D2, multigrid.prolongator(tv, dims, agg))
        Dabs = Dc.copy()
        Dabs.data = np.abs(Dabs.data)
        cs = _coarse_shape(dims, agg, nv, 3)
        x = rng.standard_normal(cs) + 1j * rng.standard_normal(cs)
        y64 = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 0).cpu().numpy()
        ysp = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 1).cpu().numpy()
        for r in range(3):
            ref = Dc @ x[r].reshape(-1)
            assert rel(y64[r].reshape(-1), ref) < 1e-12, (nv, r)
            assert np.all(np.abs(ysp[r].reshape(-1) - ref) <= u_split(2 * nv) * (Dabs @ np.abs(x[r].reshape(-1)))), (nv, r)
    ctx.close()


@pytest.mark.parametrize("dims,agg,nv", [CASES[0], CASES[2]])
def test_coarse_operator_fp64_assembly(monkeypatch, dims, agg, nv):
    """With WD_DD=0 the setup assembles D_c in FP64 arithmetic (k_assemble):
    the site block and the forward blocks, the backward ones derived from the
    gamma5c-hermiticity of D_c.  The coarse operator matches the oracle's
    P^dag D P to 1e-12 on coarse extents 2 and 1 (where forward and backward
    neighbours coincide)."""
    import torch
    from paper_2607_05157_b300 import wd_coarse_apply
    monkeypatch.setenv('WD_DD', '0')
    ctx, U, D, P = _setup(dims, agg, nv)
    Dc = multigrid.coarse_operator(D, P)
    cs = _coarse_shape(dims, agg, nv, 3)
    rng = np.random.default_rng(23)
    x = rng.standard_normal(cs) + 1j * rng.standard_normal(cs)
    y = wd_coarse_apply(ctx.h, to_dev(x), torch.empty(cs, dtype=torch.complex128, device='cuda'), 0).cpu().numpy()
    for r in range(3):
        ref = Dc @ x[r].reshape(-1)
        assert np.abs(y[r].reshape(-1) - ref).max() <= 1e-12 * np.abs(ref).max(), r
    ctx.close()
