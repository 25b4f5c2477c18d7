"""Parity of the adjoint: the link-force kernel element by element
against the oracle, the estimator gradient against the oracle's dense
per-vector computation on identical noise, the autograd path against central
finite differences (h = 1e-5, FP64) on 32 random su(3) link directions on
8^3 x 16 and 16^3 x 32, and against the dense oracle's exact gradient in the
exact probing limit on 4^4."""
import numpy as np
import pytest

import synth
from oracle import coloring, estimators, gradient, noise, solver, wilson
from tests.gpu_util import rel, to_dev

pytestmark = pytest.mark.gpu
BC = (1, 1, 1, -1)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 6, 4)])
def test_link_force_parity(dims):
    import torch
    from paper_2607_05157_b300 import Context, wd_link_force
    U = synth.gauge_field(dims, 0.5, 7)
    w, z = synth.spinors(dims, 3, 8), synth.spinors(dims, 3, 9)
    ctx = Context(dims, U, 0.13, BC)
    G = torch.empty(U.shape, dtype=torch.complex128, device='cuda')
    H = torch.empty_like(G)
    wd_link_force(ctx.h, to_dev(w), to_dev(z), G, H)
    Gr, Hr = gradient.link_force(w, z, 0.13, BC)
    assert np.abs(G.cpu().numpy() - Gr).max() < 1e-12 * np.abs(Gr).max()
    assert np.abs(H.cpu().numpy() - Hr).max() < 1e-12 * np.abs(Hr).max()
    ctx.close()


@pytest.mark.parametrize("uniform", [True, False])
def test_estimator_gradient_vs_oracle(uniform):
    """Probing d = 1 x full dilution on 4^4: G, H and dL/dkappa of
    L = Re sum_t wt[t] mean_i X_i(t) against the oracle with dense solves."""
    from paper_2607_05157_b300 import Context, WD_PROBE
    from paper_2607_05157_b300.api import trace_gradient
    dims, kappa, N, seed = (4, 4, 4, 4), 0.125, 2, 31
    U = synth.gauge_field(dims, 0.5, 10)
    ctx = Context(dims, U, kappa, BC)
    T = dims[3]
    wt = np.ones(T) if uniform else np.linspace(0.5, 2.0, T)
    dk, G, H = trace_gradient(ctx.h, WD_PROBE, 12, N, T, d=1, seed=seed, op=1, prec=1, tol=1e-12, weights=wt,
                              link_shape=U.shape)
    V = int(np.prod(dims))
    Dm = wilson.sparse_matrix(U, kappa, BC)
    Dinv = solver.dense_inverse(Dm)
    Bdiag = wilson.gamma5_full(V) * wt[wilson.timeslice_of_dof(dims)]
    nc, sigma = coloring.search(dims, 1)
    masks = estimators.probing_masks(coloring.colors(dims, sigma, nc), nc, 12)
    shape = synth.spinors(dims, 1, 0).shape[1:]
    ws, zs, dkr = [], [], 0.0
    for i in range(N):
        eta = noise.rademacher(seed, i, 12 * V)
        for m in masks:
            v = np.where(m, eta, 0).astype(complex)
            z = Dinv @ v
            w = Dinv.conj().T @ (Bdiag * v)
            zs.append(z.reshape(shape)); ws.append(w.reshape(shape))
            dkr += (np.vdot(w, z) - np.vdot(Bdiag * v, z)).real
    Gr, Hr = gradient.link_force(np.array(ws), np.array(zs), kappa, BC)
    Gr /= N; Hr /= N
    assert np.abs(G.cpu().numpy() - Gr).max() < 1e-9 * np.abs(Gr).max()
    assert np.abs(H.cpu().numpy() - Hr).max() < 1e-9 * np.abs(Hr).max()
    assert abs(dk - dkr / (N * kappa)) < 1e-9 * abs(dkr / (N * kappa))
    ctx.close()


def _exp_pair(T, h):
    """exp(+i h T) and exp(-i h T) on every link for Hermitian T, from one
    eigendecomposition per link."""
    lam, V = np.linalg.eigh(T)
    Vh = np.conj(np.swapaxes(V, -1, -2))
    return tuple(np.einsum('...ab,...b,...bc->...ac', V, np.exp(1j * s * h * lam), Vh) for s in (1.0, -1.0))


@pytest.mark.parametrize("dims", [(8, 8, 8, 16), (16, 16, 16, 32)])
def test_autograd_vs_finite_differences(dims):
    """The differentiation workload (kappa 0.125, probing d = 2 x 12
    dilution, gamma5) on 8^3 x 16 and 16^3 x 32: the autograd gradient against
    central differences in FP64 along 32 random su(3) link directions
    (U -> exp(i h T) U, h = 1e-5) and in kappa, relative agreement 1e-6."""
    import torch
    from paper_2607_05157_b300 import Context, WD_PROBE
    from paper_2607_05157_b300.autograd import TraceFn
    kappa, seed, N = 0.125, 41, 1
    U = synth.gauge_field(dims, 0.5, 1005)
    ctx = Context(dims, U, kappa, BC)
    Ut = to_dev(U).requires_grad_(True)
    kt = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    wt = torch.linspace(0.5, 1.5, dims[3], dtype=torch.float64, device='cuda')
    args = (ctx, WD_PROBE, 12, N, 2, seed, 1, 1e-13)
    L = (TraceFn.apply(kt, Ut, *args) * wt).sum()
    L.backward()
    gU = Ut.grad.cpu().numpy()

    def Lval(Uh, k):
        with torch.no_grad():
            return float((TraceFn.apply(torch.tensor(k, dtype=torch.float64), to_dev(Uh), *args) * wt).sum())
    h = 1e-5
    for j in range(32):
        Tj = synth.su3_algebra(dims, 500 + j)
        Ep, Em = _exp_pair(Tj, h)
        fd = (Lval(np.einsum('...ab,...bc->...ac', Ep, U), kappa) -
              Lval(np.einsum('...ab,...bc->...ac', Em, U), kappa)) / (2 * h)
        Delta = 1j * np.einsum('...ab,...bc->...ac', Tj, U)
        an = np.sum((np.conj(gU) * Delta)).real          # Re sum conj(grad) * Delta
        assert abs(fd - an) <= 1e-6 * abs(an), (j, fd, an)
    fdk = (Lval(U, kappa + 1e-6) - Lval(U, kappa - 1e-6)) / 2e-6
    assert abs(fdk - float(kt.grad)) <= 1e-6 * abs(fdk)
    ctx.close()


def test_autograd_exact_probing_limit_4x4x4x4():
    """Every dof its own vector -- time dilution x the 3D colouring of a 4^3
    timeslice at distance 6 (64 colours: every site of a timeslice its own) x
    12-fold spin-colour dilution -- makes the probing estimate exact for any
    noise: the estimate equals the dense trace per timeslice, and the autograd
    gradient of L = sum_t w_t O(t) equals the exact derivative
    -tr(B D^{-1} dD D^{-1}) (B = g5 weighted per timeslice) in random su(3)
    directions and in kappa, from the dense oracle."""
    import torch
    from paper_2607_05157_b300 import Context, WD_PROBE, WD_DIL_TIME, WD_COLOR_3D
    from paper_2607_05157_b300.autograd import TraceFn
    dims, kappa = (4, 4, 4, 4), 0.125
    U = synth.gauge_field(dims, 0.5, 1005)
    ctx = Context(dims, U, kappa, BC)
    Ut = to_dev(U).requires_grad_(True)
    kt = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    w_np = np.linspace(0.5, 1.5, dims[3])
    wt = torch.tensor(w_np, dtype=torch.float64, device='cuda')
    args = (ctx, WD_PROBE, 12 | WD_DIL_TIME | WD_COLOR_3D, 1, 6, 77, 1, 1e-13)
    est = TraceFn.apply(kt, Ut, *args)
    D = wilson.sparse_matrix(U, kappa, BC)
    Dinv = solver.dense_inverse(D)
    exact = solver.exact_traces(Dinv, dims, True).real
    assert np.abs(est.detach().cpu().numpy() - exact).max() <= 1e-8 * max(1.0, np.abs(exact).max())
    (est * wt).sum().backward()
    gU = Ut.grad.cpu().numpy()
    V = int(np.prod(dims))
    Bdiag = wilson.gamma5_full(V) * w_np[wilson.timeslice_of_dof(dims)]
    for j in range(4):
        Delta = 1j * np.einsum('...ab,...bc->...ac', synth.su3_algebra(dims, 700 + j), U)
        an = np.sum(np.conj(gU) * Delta).real
        ex = gradient.exact_derivative(Dinv, Bdiag, gradient.hopping_derivative(Delta, kappa, BC)).real
        assert abs(an - ex) <= 1e-8 * abs(ex), (j, an, ex)
    import scipy.sparse as sp
    dD_dk = (D - sp.identity(12 * V, dtype=np.complex128, format='csr')) / kappa      # D = 1 - kappa H: dD/dk = -H
    exk = gradient.exact_derivative(Dinv, Bdiag, dD_dk).real
    assert abs(float(kt.grad) - exk) <= 1e-8 * abs(exk)
    ctx.close()
