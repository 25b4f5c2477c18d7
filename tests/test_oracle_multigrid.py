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


# ---- MLMC combined with probing (Sec. 6 outlook) and the N_l allocation (Eq. 6)

def test_mlmc_allocation_hand_example_and_brute_force():
    """Eq. 6 on V = (4, 1), C = (1, 4), eps = 1: sum sqrt(V C) = 4, so
    N = (sqrt(4) * 4, sqrt(1/4) * 4) = (8, 2); variance 4/8 + 1/2 = 1 = eps^2.
    Brute force over integer pairs finds the same minimum cost 16."""
    Nc, Ni = estimators.mlmc_allocation([4.0, 1.0], [1.0, 4.0], 1.0)
    assert np.allclose(Nc, [8.0, 2.0], rtol=0, atol=1e-12) and list(Ni) == [8, 2]
    best = min((n1 + 4 * n2, n1, n2) for n1 in range(1, 60) for n2 in range(1, 60) if 4 / n1 + 1 / n2 <= 1)
    assert best == (16, 8, 2)


def test_mlmc_allocation_is_the_constrained_minimum():
    """The continuous N_l meet the variance target exactly, and every other
    point on the constraint surface sum V_l / N_l = eps^2 costs more."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        L = int(rng.integers(2, 5))
        V = rng.uniform(0.1, 10.0, L)
        C = rng.uniform(0.1, 10.0, L)
        eps = float(rng.uniform(0.05, 1.0))
        Nc, Ni = estimators.mlmc_allocation(V, C, eps)
        assert abs(np.sum(V / Nc) - eps ** 2) < 1e-12 * eps ** 2
        cost = np.sum(Nc * C)
        for _ in range(50):
            # another feasible point: scale a random positive vector onto the constraint
            N = Nc * np.exp(rng.normal(0, 0.3, L))
            N *= np.sum(V / N) / eps ** 2
            assert abs(np.sum(V / N) - eps ** 2) < 1e-9 * eps ** 2
            assert np.sum(N * C) >= cost * (1 - 1e-12)
        # rounding up keeps the variance within the target
        assert np.sum(V / Ni) <= eps ** 2 * (1 + 1e-12) and np.all(Ni >= 1)


@pytest.fixture(scope='module')
def mg_probe():
    dims, agg, nv = (2, 2, 2, 4), (2, 2, 2, 2), 3
    U = synth.gauge_field(dims, 0.4, 1010)
    D = wilson.sparse_matrix(U, 0.12, BC_AP)
    P = multigrid.prolongator(synth.test_vectors(dims, nv, 5), dims, agg)
    Dinv = solver.dense_inverse(D)
    Dcinv = solver.dense_inverse(multigrid.coarse_operator(D, P))
    return dims, U, D, P, Dinv, Dcinv


@pytest.mark.parametrize("time_dilution", [False, True])
def test_mlmc2_probe_level1_is_difference_of_probing(mg_probe, time_dilution):
    """Level 1 of the combined estimator is linear in the operator: each
    sample equals the probing sample of D^{-1} minus the probing sample of
    P D_c^{-1} P^dag on the same vectors (probing pinned separately)."""
    from oracle import coloring
    dims, U, D, P, Dinv, Dcinv = mg_probe
    Pd = P.toarray()
    nc, sigma = coloring.search(dims, 1)
    col = coloring.colors(dims, sigma, nc)
    X1, X2 = estimators.mlmc2_probe(lambda v: Dinv @ v, lambda v: Dcinv @ v, P, dims, 7, 3, 4, True, col, nc,
                                    12, time_dilution)
    coarse = Pd @ Dcinv @ Pd.conj().T
    if time_dilution:
        # each timeslice's vectors form their own probing set: sum over t of
        # probing with the masks restricted to t
        ts = wilson.timeslice_of_dof(dims)
        ref = np.zeros_like(X1)
        from oracle import noise
        for i in range(3):
            eta = noise.rademacher(7, i, 12 * int(np.prod(dims)))
            for m in estimators.probing_masks(col, nc, 12):
                for t in range(dims[3]):
                    v = np.where(m & (ts == t), eta, 0).astype(complex)
                    ref[i] += estimators.contract(v, Dinv @ v - coarse @ v, dims, True)
    else:
        ref = (estimators.probing(lambda v: Dinv @ v, dims, 7, 3, True, col, nc, 12) -
               estimators.probing(lambda v: coarse @ v, dims, 7, 3, True, col, nc, 12))
    assert np.abs(X1 - ref).max() < 1e-12 * np.abs(ref).max()
    _, R2 = estimators.mlmc2(lambda v: Dinv @ v, lambda v: Dcinv @ v, P, dims, 7, 0, 4, True)
    assert np.array_equal(X2, R2)


@pytest.mark.parametrize("time_dilution", [False, True])
def test_mlmc2_probe_exact_when_every_dof_is_its_own_vector(time_dilution):
    """With a colouring that gives every site its own colour (distance 4 on
    a 2^4 torus) and full spin-colour dilution, every probing vector has one
    nonzero entry, so level 1 equals tr[B M_1(t, t)] exactly for any noise
    (Eq. 10: M_1 = D^{-1} - P D_c^{-1} P^dag)."""
    from oracle import coloring
    dims = (2, 2, 2, 2)
    U = synth.gauge_field(dims, 0.4, 1011)
    D = wilson.sparse_matrix(U, 0.12, BC_AP)
    P = multigrid.prolongator(synth.test_vectors(dims, 2, 6), dims, (2, 2, 2, 2))
    Dinv = solver.dense_inverse(D)
    Dcinv = solver.dense_inverse(multigrid.coarse_operator(D, P))
    nc, sigma = coloring.search(dims, 4)
    assert nc == 16
    col = coloring.colors(dims, sigma, nc)
    X1, _ = estimators.mlmc2_probe(lambda v: Dinv @ v, lambda v: Dcinv @ v, P, dims, 11, 2, 1, True, col, nc,
                                   12, time_dilution)
    Pd = P.toarray()
    M = Dinv - Pd @ Dcinv @ Pd.conj().T
    d = wilson.gamma5_full(int(np.prod(dims))) * np.diag(M)
    ts = wilson.timeslice_of_dof(dims)
    exact = np.array([d[ts == t].sum() for t in range(dims[3])])
    for i in range(2):
        assert np.abs(X1[i] - exact).max() < 1e-12 * np.abs(exact).max()


def test_mlmc2_probe_coarse_level_reduces_to_plain_and_exact_limit(mg_probe):
    """Level 2 with coarse probing: one colour and no dilution is the plain
    coarse estimator of mlmc2 (pinned separately); every coarse site its own
    colour with full coarse-dof dilution gives tr[B P D_c^{-1} P^dag (t, t)]
    exactly for any noise."""
    from oracle import coloring
    dims, U, D, P, Dinv, Dcinv = mg_probe
    cd = multigrid.coarse_dims(dims, (2, 2, 2, 2))
    Vc = int(np.prod(cd))
    ncd = P.shape[1]
    nc, sigma = coloring.search(dims, 1)
    col = coloring.colors(dims, sigma, nc)
    solve, solve_c = (lambda v: Dinv @ v), (lambda v: Dcinv @ v)
    _, X2a = estimators.mlmc2_probe(solve, solve_c, P, dims, 8, 0, 3, True, col, nc, 1,
                                    coarse_col=np.zeros(Vc, int), coarse_nc=1, coarse_dil=1)
    _, X2b = estimators.mlmc2(solve, solve_c, P, dims, 8, 0, 3, True)
    assert np.abs(X2a - X2b).max() < 1e-13 * np.abs(X2b).max()
    _, X2 = estimators.mlmc2_probe(solve, solve_c, P, dims, 8, 0, 2, True, col, nc, 1,
                                   coarse_col=np.arange(Vc), coarse_nc=Vc, coarse_dil=ncd // Vc)
    Pd = P.toarray()
    d = wilson.gamma5_full(int(np.prod(dims))) * np.diag(Pd @ Dcinv @ Pd.conj().T)
    ts = wilson.timeslice_of_dof(dims)
    exact = np.array([d[ts == t].sum() for t in range(dims[3])])
    for i in range(2):
        assert np.abs(X2[i] - exact).max() < 1e-12 * np.abs(exact).max()


# ---- three levels ----------------------------------------------------------

@pytest.fixture(scope='module')
def mg3():
    dims, agg, nv = (4, 4, 4, 4), (2, 2, 2, 2), 6
    U = synth.gauge_field(dims, 0.3, 1030)
    D = wilson.sparse_matrix(U, 0.12, BC_AP)
    P1 = multigrid.prolongator(synth.test_vectors(dims, nv, 31), dims, agg)
    D2 = multigrid.coarse_operator(D, P1)
    cd = multigrid.coarse_dims(dims, agg)
    rng = np.random.default_rng(32)
    nv2 = 6
    tv2 = rng.standard_normal((nv2, D2.shape[0])) + 1j * rng.standard_normal((nv2, D2.shape[0]))
    P2 = multigrid.prolongator_coarse(tv2, cd, (2, 2, 2, 2), nv)
    D3 = multigrid.coarse_operator(D2, P2)
    return dims, D, P1, D2, P2, D3


def test_three_level_transfer_and_telescoping(mg3):
    """P_2^dag P_2 = I; P_2 keeps the chirality halves (gamma5 of level 2
    maps to gamma5 of level 3); the level split telescopes:
    tr(M_1) + tr(P_1 M_2 P_1^dag) + tr(P_1 P_2 D_3^{-1} P_2^dag P_1^dag) = tr(D^{-1})
    (Eqs. 10-11 with L = 3); the second oblique projector is idempotent."""
    dims, D, P1, D2, P2, D3 = mg3
    PP = (P2.conj().T @ P2).toarray()
    assert np.abs(PP - np.eye(PP.shape[0])).max() < 1e-13
    g2 = multigrid.gamma5_coarse(6, P1.shape[1] // 12)
    g3 = multigrid.gamma5_coarse(6, P2.shape[1] // 12)
    assert np.abs(g2[:, None] * P2.toarray() - P2.toarray() * g3[None, :]).max() < 1e-14
    Dinv = solver.dense_inverse(D)
    D2inv = solver.dense_inverse(D2)
    D3inv = solver.dense_inverse(D3)
    A1, A2 = P1.toarray(), P2.toarray()
    M1 = Dinv - A1 @ D2inv @ A1.conj().T
    M2 = D2inv - A2 @ D3inv @ A2.conj().T
    total = np.trace(M1) + np.trace(A1 @ M2 @ A1.conj().T) + np.trace(A1 @ A2 @ D3inv @ A2.conj().T @ A1.conj().T)
    assert abs(total - np.trace(Dinv)) < 1e-12 * abs(np.trace(Dinv))
    Pi = A2 @ D3inv @ (A2.conj().T @ D2.toarray())
    assert np.abs(Pi @ Pi - Pi).max() < 1e-10 * np.abs(Pi).max()


def test_three_level_nine_point_sparsity(mg3):
    """D_3 couples each level-3 site only to itself and its nearest
    neighbours (a 9-point block stencil like D_2)."""
    dims, D, P1, D2, P2, D3 = mg3
    cd3 = multigrid.coarse_dims(multigrid.coarse_dims(dims, (2, 2, 2, 2)), (2, 2, 2, 2))
    assert cd3 == (1, 1, 1, 1) and D3.shape == (12, 12)


def test_mlmc3_unbiased_and_levels(mg3):
    """Each level's sample mean is within 5 sigma of its exact trace, and the
    three exact level traces sum to tr(D^{-1}) (B = 1)."""
    dims, D, P1, D2, P2, D3 = mg3
    Dinv = solver.dense_inverse(D)
    D2inv = solver.dense_inverse(D2)
    D3inv = solver.dense_inverse(D3)
    X1, X2, X3 = estimators.mlmc3(lambda v: Dinv @ v, lambda v: D2inv @ v, lambda v: D3inv @ v, P1, P2, dims, 5,
                                  48, 96, 256, False)
    A1, A2 = P1.toarray(), P2.toarray()
    exact = [np.trace(Dinv - A1 @ D2inv @ A1.conj().T),
             np.trace(D2inv - A2 @ D3inv @ A2.conj().T),     # = tr(P_1 M_2 P_1^dag) since P_1^dag P_1 = I
             np.trace(D3inv)]
    for Xl, ex, M in ((X1, exact[0], Dinv - A1 @ D2inv @ A1.conj().T),
                      (X2, exact[1], D2inv - A2 @ D3inv @ A2.conj().T), (X3, exact[2], D3inv)):
        _, _, m, v = estimators.mean_and_variance(Xl)
        V = estimators.hutchinson_variance(M)
        assert abs(m - ex) < 5 * np.sqrt(V / Xl.shape[0]) + 1e-12
    assert abs(sum(exact) - np.trace(Dinv)) < 1e-12 * abs(np.trace(Dinv))


# ---- test vectors by inverse iteration (Sec. 2's setup) ---------------------

def _free_dinv(v, dims, kappa, bc):
    """D^{-1} v for U = 1 from the momentum-space closed form
    D(p)^{-1} = (a - i gamma.b) / (a^2 + |b|^2) (independent of the stencil
    and of the solver): twist the antiperiodic directions, FFT, multiply,
    inverse FFT, untwist."""
    from oracle.gamma import GAMMA, ID4
    w = np.asarray(v, np.complex128)
    twist = np.ones(w.shape[:4], np.complex128)
    ps = []
    for mu, L in enumerate(dims):
        ax = 3 - mu                                  # axes (t, z, y, x)
        k = np.arange(L)
        ps.append((2 * np.pi * k + (np.pi if bc[mu] == -1 else 0.0)) / L)
        if bc[mu] == -1:
            shp = [1, 1, 1, 1]
            shp[ax] = L
            twist = twist * np.exp(1j * np.pi * k / L).reshape(shp)
    wt = np.fft.fftn(w / twist[..., None, None], axes=(0, 1, 2, 3))
    pt, pz, py, px = np.meshgrid(ps[3], ps[2], ps[1], ps[0], indexing='ij')
    P = [px, py, pz, pt]
    a = 1 - 2 * kappa * sum(np.cos(p) for p in P)
    bs = [2 * kappa * np.sin(p) for p in P]
    den = a * a + sum(b * b for b in bs)
    M = np.einsum('...,st->...st', a / den, ID4)
    for mu in range(4):
        M = M - 1j * np.einsum('...,st->...st', bs[mu] / den, GAMMA[mu])
    yt = np.einsum('tzyxsr,tzyxrc->tzyxsc', M, wt)
    return np.fft.ifftn(yt, axes=(0, 1, 2, 3)) * twist[..., None, None]


def test_free_dinv_helper_inverts_the_stencil():
    dims, kappa, bc = (4, 4, 2, 6), 0.12, (1, 1, 1, -1)
    U = synth.unit_gauge(dims)
    v = synth.spinors(dims, 1, 3)[0]
    y = _free_dinv(v, dims, kappa, bc)
    assert np.abs(wilson.apply(U, y, kappa, bc) - v).max() < 1e-12 * np.abs(v).max()


def test_test_vectors_free_field_closed_form():
    """Two inverse iterations on U = 1 equal D^{-2} eta / ||D^{-2} eta|| with
    D^{-1} from momentum space, for the Rademacher starts of samples 2^22 + k."""
    from oracle import noise
    dims, kappa, bc, seed = (4, 4, 4, 4), 0.12, (1, 1, 1, -1), 7
    U = synth.unit_gauge(dims)
    tv = multigrid.test_vectors(lambda v: wilson.apply(U, v, kappa, bc), dims, 2, 2, seed)
    shape = (dims[3], dims[2], dims[1], dims[0], 4, 3)
    for k in range(2):
        v = noise.rademacher(seed, (1 << 22) + k, 12 * 256).reshape(shape)
        for _ in range(2):
            v = _free_dinv(v, dims, kappa, bc)
            v = v / np.linalg.norm(v)
        assert np.abs(tv[k] - v).max() < 1e-9
    # no iterations: the starts themselves
    tv0 = multigrid.test_vectors(lambda v: wilson.apply(U, v, kappa, bc), dims, 1, 0, seed)
    assert np.array_equal(tv0[0].real.reshape(-1), noise.rademacher(seed, 1 << 22, 12 * 256))


def test_test_vectors_converge_to_the_smallest_eigenspace():
    """Inverse iteration converges to the invariant subspace of the eigenvalues
    of D of smallest modulus (a complex-conjugate pair for this gamma5-hermitian
    D); the eigen-decomposition is numpy's dense one."""
    dims, kappa, bc = (2, 2, 2, 2), 0.16, (1, 1, 1, -1)
    U = synth.gauge_field(dims, 0.5, 11)
    Dm = wilson.sparse_matrix(U, kappa, bc).toarray()
    lam, E = np.linalg.eig(Dm)
    mod = np.abs(lam)
    order = np.argsort(mod)
    m0 = mod[order[0]]
    low = order[mod[order] <= m0 * (1 + 1e-9)]
    nxt = mod[order[len(low)]]
    ratio = m0 / nxt
    assert ratio < 0.95
    iters = int(np.ceil(np.log(1e-11) / np.log(ratio)))
    tv = multigrid.test_vectors(lambda v: wilson.apply(U, v, kappa, bc), dims, 1, iters, 5)
    v = tv[0].reshape(-1)
    B = E[:, low]
    coef = np.linalg.lstsq(B, v, rcond=None)[0]
    assert np.linalg.norm(v - B @ coef) < 1e-7
    assert abs(np.linalg.norm(v) - 1.0) < 1e-14
