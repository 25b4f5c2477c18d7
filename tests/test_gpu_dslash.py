"""Parity of the fine Wilson stencil (through wd_apply) with the oracle,
element by element, FP64 / FP32 / BF16, D and D^dag, ragged RHS counts."""
import numpy as np
import pytest

import synth
from oracle import wilson
from tests.gpu_util import rel, to_dev

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)
# normwise bounds: FP64 from the benchmark spec's tolerance; double-float (3): inputs
# split to 47 bits, every product and sum exact up to terms of 2^-48 relative,
# ~100 of them per output -> a few 1e-14, bound 1e-12.  FP32 and BF16 are held
# element by element to ELEM_U[prec] * abs_stencil_bound (below).
TOL = {0: 1e-13, 1: 3e-6, 2: 2e-2, 3: 1e-12}
# Element-wise error bound factors u_eff, |y - ref| <= u_eff * B with B the
# stencil applied to absolute values.  FP32 (input already FP32, the reference
# computed from the same FP32 input): the FP32 copy of each link (2^-24) and
# at most ~20 rounded operations along any product-and-sum chain of an output
# (spin projection, SU(3) row, reconstruction, 8 directions, the final
# a w + b H psi): 24 * 2^-24.  BF16 storage of links and input (8 significant
# bits, unit roundoff 2^-8 each): 2 * 2^-8 + 2^-16 per product plus the FP32
# arithmetic.
ELEM_U = {1: 24 * 2.0 ** -24, 2: 2 * 2.0 ** -8 + 2.0 ** -16 + 24 * 2.0 ** -24}


def abs_stencil_bound(U, psi, kappa):
    """B = |psi| + kappa sum_mu [ |1 -/+ g_mu| (|U_mu(x)| |psi(x+mu)|)
    + |1 +/- g_mu| (|U_mu(x-mu)|^T |psi(x-mu)|) ] element by element (complex
    moduli of every entry; the same for D and D^dag).  Every term of an output
    component of D psi is bounded by the matching term of B, so a kernel's
    rounding error is a small multiple of B -- and a dropped or wrong term is
    a change of order B itself."""
    from oracle.gamma import GAMMA, ID4
    a = np.abs(psi)
    out = a.copy()
    ax = {0: -3, 1: -4, 2: -5, 3: -6}          # x, y, z, t axes of (..., T, Z, Y, X, 4, 3)
    for mu in range(4):
        G = np.abs(ID4 + GAMMA[mu])           # |1 + g| = |1 - g| entry by entry
        Uf = np.abs(U[mu])
        Ub = np.roll(Uf, 1, axis=ax[mu] + 2)  # |U_mu(x - mu)|
        fwd = np.einsum('...ab,...sb->...sa', Uf, np.roll(a, -1, axis=ax[mu]))
        bwd = np.einsum('...ba,...sb->...sa', Ub, np.roll(a, 1, axis=ax[mu]))
        out = out + kappa * np.einsum('st,...tc->...sc', G, fwd + bwd)
    return out


def assert_elementwise(y, ref, bound, u, what=''):
    err = np.abs(y - ref)
    worst = (err / (u * bound + 1e-300)).max()
    assert worst <= 1.0, (what, worst)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 6, 8), (6, 2, 4, 2)])
@pytest.mark.parametrize("nrhs", [1, 3, 5])
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_parity(dims, nrhs, prec, dagger):
    import torch
    from paper_2607_05157_b300 import Context
    U = synth.gauge_field(dims, 0.5, 1002)
    kappa = 0.125
    psi = synth.spinors(dims, nrhs, 31)
    ctx = Context(dims, U, kappa, BC)
    dt = torch.complex128 if prec in (0, 3) else torch.complex64
    if prec in (1, 2):
        psi = psi.astype(np.complex64).astype(np.complex128)    # the input the kernel sees
    y = ctx.apply(to_dev(psi, dt), prec=prec, dagger=dagger).cpu().numpy()
    f = wilson.apply_dagger if dagger else wilson.apply
    ref = f(U, psi, kappa, BC)
    for r in range(nrhs):
        assert rel(y[r], ref[r]) < TOL[prec], (r, rel(y[r], ref[r]))
    if prec in (1, 2):
        assert_elementwise(y, ref, abs_stencil_bound(U, psi, kappa), ELEM_U[prec], (dims, nrhs, prec, dagger))
    if prec == 0:
        assert np.abs(y - ref).max() < 1e-13 * np.abs(ref).max()
    if prec == 3:
        assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max()
    ctx.close()


@pytest.mark.parametrize("scale", [1e-25, 1e-8, 1.0, 1e25])
def test_apply_double_float_range(scale):
    """Double-float stencil over the input range it supports (2^-103 .. 2^127):
    relative accuracy independent of the scale; exact zeros (time-diluted
    sources are zero off their timeslice) stay zero."""
    import torch
    from paper_2607_05157_b300 import Context, WD_FP64_DD
    dims = (4, 4, 4, 8)
    U = synth.gauge_field(dims, 0.5, 1004)
    psi = synth.spinors(dims, 2, 77) * scale
    psi[1, 2:] = 0.0          # rhs 1: zero on timeslices 2..7
    ctx = Context(dims, U, 0.125, BC)
    y = ctx.apply(to_dev(psi), prec=WD_FP64_DD).cpu().numpy()
    ref = wilson.apply(U, psi, 0.125, BC)
    for r in range(2):
        assert rel(y[r], ref[r]) < TOL[3], (scale, r, rel(y[r], ref[r]))
    # D = 1 - k H: no output outside timeslices 1..3 for rhs 1 except from t = 0, 1
    assert np.all(y[1, 3:7] == 0.0)
    ctx.close()


@pytest.mark.parametrize("variant", ["1", "2:64", "11", "12:64"])
@pytest.mark.parametrize("dagger", [False, True])
def test_apply_double_float_variants(monkeypatch, variant, dagger):
    """Every launch shape of the double-float stencil (scalar R = 1, 2; packed
    f32x2 R = 1, 2) against the oracle, on a ragged RHS count and lattice."""
    import torch
    from paper_2607_05157_b300 import Context, WD_FP64_DD
    monkeypatch.setenv('WD_DD_R', variant)
    dims = (2, 4, 6, 8)
    U = synth.gauge_field(dims, 0.5, 1005)
    psi = synth.spinors(dims, 5, 78)
    ctx = Context(dims, U, 0.125, BC)
    y = ctx.apply(to_dev(psi), prec=WD_FP64_DD, dagger=dagger).cpu().numpy()
    f = wilson.apply_dagger if dagger else wilson.apply
    ref = f(U, psi, 0.125, BC)
    for r in range(5):
        assert rel(y[r], ref[r]) < TOL[3], (variant, r, rel(y[r], ref[r]))
    assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max()
    ctx.close()


def test_apply_double_float_vs_fp64_and_fp32():
    """The double-float stencil is at least 10^4 times closer to the FP64
    result than the FP32 stencil on the same input (8^3 x 16, 16 RHS)."""
    import torch
    from paper_2607_05157_b300 import Context, WD_FP64_DD
    dims = (8, 8, 8, 16)
    U = synth.gauge_field(dims, 0.5, 1002)
    psi = synth.spinors(dims, 16, 9)
    ctx = Context(dims, U, 0.125, BC)
    y64 = ctx.apply(to_dev(psi), prec=0).cpu().numpy()
    ydd = ctx.apply(to_dev(psi), prec=WD_FP64_DD).cpu().numpy()
    y32 = ctx.apply(to_dev(psi, torch.complex64), prec=1).cpu().numpy()
    e_dd = max(rel(ydd[r], y64[r]) for r in range(16))
    e_32 = max(rel(y32[r], y64[r]) for r in range(16))
    assert e_dd < 1e-12 and e_dd * 1e4 < e_32, (e_dd, e_32)
    ctx.close()


def test_apply_full_size_sampled():
    """16^3 x 32 (the probing workload), 12 RHS in FP32, FP64 on 2: compared on
    every site of two RHS against the oracle."""
    import torch
    from paper_2607_05157_b300 import Context
    dims = (16, 16, 16, 32)
    U = synth.gauge_field(dims, 0.5, 1003)
    psi = synth.spinors(dims, 12, 5).astype(np.complex64).astype(np.complex128)
    ctx = Context(dims, U, 0.13, BC)
    y32 = ctx.apply(to_dev(psi, torch.complex64), prec=1).cpu().numpy()
    y64 = ctx.apply(to_dev(psi[:2]), prec=0).cpu().numpy()
    for r in (0, 11):
        ref = wilson.apply(U, psi[r], 0.13, BC)
        assert rel(y32[r], ref) < TOL[1]
        assert_elementwise(y32[r], ref, abs_stencil_bound(U, psi[r], 0.13), ELEM_U[1], r)
        if r < 2:
            assert rel(y64[r], ref) < TOL[0]
    ref1 = wilson.apply(U, psi[1], 0.13, BC)
    assert rel(y64[1], ref1) < TOL[0]
    ctx.close()


def test_free_field_plane_wave():
    """U = 1: D e^{ipx} u = (a + i gamma.b) e^{ipx} u, a property of the
    operator that holds at any size (checked on 8^3 x 16)."""
    import torch
    from paper_2607_05157_b300 import Context
    from oracle import freefield, gamma
    dims = (8, 8, 8, 16)
    X, Y, Z, T = dims
    kappa = 0.125
    ctx = Context(dims, synth.unit_gauge(dims), kappa, BC)
    k = (1, 2, 3, 0)
    p = [freefield.momenta(L, b)[kk] for L, b, kk in zip(dims, BC, k)]
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing='ij')
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    u = np.random.default_rng(0).standard_normal((4, 3)) + 0j
    psi = (phase[..., None, None] * u)[None]
    out = ctx.apply(to_dev(psi)).cpu().numpy()
    a = 1 - 2 * kappa * sum(np.cos(q) for q in p)
    Mp = a * np.eye(4) + 1j * sum(2 * kappa * np.sin(q) * g for q, g in zip(p, gamma.GAMMA))
    ref = phase[..., None, None] * (Mp @ u)[None]
    assert np.abs(out[0] - ref).max() < 1e-13
    ctx.close()
