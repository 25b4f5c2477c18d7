"""Parity of the adjoint (row a10): the link-force kernel element by element
against the oracle, the estimator gradient against the oracle's dense
per-vector computation on identical noise, and the autograd path against
central finite differences (h = 1e-5, FP64) on random su(3) link directions."""
import numpy as np
import pytest
import scipy.linalg as sla

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


def _expm_links(T, h):
    return np.array([sla.expm(1j * h * t) for t in T.reshape(-1, 3, 3)]).reshape(T.shape)


@pytest.mark.parametrize("dims", [(8, 8, 8, 16)])
def test_autograd_vs_finite_differences(dims):
    """The differentiation workload on 8^3 x 16 (kappa 0.125, probing d = 2,
    gamma5): autograd gradient vs central differences in FP64 along 8 random
    su(3) link directions and in kappa, relative agreement 1e-6."""
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
    for j in range(8):
        Tj = synth.su3_algebra(dims, 500 + j)
        Up = np.einsum('...ab,...bc->...ac', _expm_links(Tj, h), U)
        Um = np.einsum('...ab,...bc->...ac', _expm_links(Tj, -h), U)
        fd = (Lval(Up, kappa) - Lval(Um, kappa)) / (2 * h)
        Delta = 1j * np.einsum('...ab,...bc->...ac', Tj, U)
        an = np.sum((np.conj(gU) * Delta)).real          # Re sum conj(grad) * Delta
        assert abs(fd - an) <= 1e-6 * abs(an), (j, fd, an)
    fdk = (Lval(U, kappa + 1e-6) - Lval(U, kappa - 1e-6)) / 2e-6
    assert abs(fdk - float(kt.grad)) <= 1e-6 * abs(fdk)
    ctx.close()
