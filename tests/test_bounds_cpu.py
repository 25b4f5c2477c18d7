"""The element-wise error bounds the GPU parity tests use, checked on the CPU
with the oracle: an operand rounding of the kind the kernels do (BF16 storage,
emulated here) stays inside the bound, and a planted mistake in the oracle's
output -- one hop term dropped at one site, one coarse block dropped at one
coarse site, or one remainder product of the BF16-pair form dropped --
breaks it."""
import numpy as np

import synth
from oracle import multigrid, wilson
from tests.test_gpu_dslash import ELEM_U, abs_stencil_bound
from tests.test_gpu_multigrid import REL_SPLIT, U_SPLIT, U_TC, _coarse_abs_bound, _coarse_nbr

BC = (1, 1, 1, -1)


def _bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    def one(v):
        u = np.ascontiguousarray(v, np.float32).view(np.uint32).astype(np.uint64)
        u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
        return u.astype(np.uint32).view(np.float32).astype(np.float64)
    return one(a.real) + 1j * one(a.imag)


def test_fine_bound_holds_for_bf16_operands_and_catches_a_dropped_hop():
    dims, kappa = (4, 4, 4, 6), 0.125
    U = synth.gauge_field(dims, 0.5, 1002)
    psi = synth.spinors(dims, 1, 31)[0].astype(np.complex64).astype(np.complex128)
    ref = wilson.apply(U, psi, kappa, BC)
    B = abs_stencil_bound(U, psi, kappa)
    assert np.all(np.abs(ref) <= B * (1 + 1e-12))            # triangle inequality
    y16 = wilson.apply(_bf16(U), _bf16(psi), kappa, BC)       # BF16 storage, exact arithmetic
    assert np.all(np.abs(y16 - ref) <= ELEM_U[2] * B)
    Ubad = U.copy()
    Ubad[0, 2, 1, 3, 1] = 0.0                                 # one link: drops two hop terms
    ybad = wilson.apply(Ubad, psi, kappa, BC)
    assert np.any(np.abs(ybad - ref) > ELEM_U[1] * B)
    assert np.any(np.abs(ybad - ref) > ELEM_U[2] * B)


def _coarse_case():
    dims, agg, nv = (6, 6, 6, 6), (2, 2, 2, 2), 6
    cd = (3, 3, 3, 3)
    U = synth.gauge_field(dims, 0.5, 1004)
    P = multigrid.prolongator(synth.test_vectors(dims, nv, 77), dims, agg)
    Dc = multigrid.coarse_operator(wilson.sparse_matrix(U, 0.13, BC), P).toarray()
    ncd, Vc = 2 * nv, 81
    nbr = _coarse_nbr(cd)
    A = np.empty((Vc, 9, ncd, ncd), np.complex128)
    for X in range(Vc):
        for b in range(9):
            A[X, b] = Dc[X * ncd:(X + 1) * ncd, nbr[X, b] * ncd:(nbr[X, b] + 1) * ncd]
    # the 9 blocks are D_c's whole row: nothing outside them
    mask = np.zeros_like(Dc, bool)
    for X in range(Vc):
        for b in range(9):
            mask[X * ncd:(X + 1) * ncd, nbr[X, b] * ncd:(nbr[X, b] + 1) * ncd] = True
    assert np.all(Dc[~mask] == 0)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((Vc, ncd)) + 1j * rng.standard_normal((Vc, ncd))
    return Dc, A, nbr, x


def test_coarse_bound_holds_for_bf16_operands_and_catches_a_dropped_block():
    Dc, A, nbr, x = _coarse_case()
    Vc, ncd = x.shape
    ref = (Dc @ x.reshape(-1)).reshape(Vc, ncd)
    B = _coarse_abs_bound(A, nbr, x)
    y16 = (_bf16(Dc) @ _bf16(x).reshape(-1)).reshape(Vc, ncd)
    assert np.all(np.abs(y16 - ref) <= U_TC * B)
    ybad = ref.copy()
    ybad[17] -= A[17, 3] @ x[nbr[17, 3]]                      # one neighbour block dropped at one site
    assert np.any(np.abs(ybad - ref) > U_TC * B)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_coarse_bound_holds_for_bf16_pairs_and_catches_a_dropped_remainder():
    """BF16-pair operands (v = hi + lo, lo the BF16 rounding of v - hi; the
    input first rounded to FP32) multiplied as hi hi + lo hi + hi lo: inside
    U_SPLIT element by element and REL_SPLIT normwise.  Dropping either
    remainder product, or a block, breaks them."""
    Dc, A, nbr, x = _coarse_case()
    Vc, ncd = x.shape
    ref = (Dc @ x.reshape(-1)).reshape(Vc, ncd)
    B = _coarse_abs_bound(A, nbr, x)
    x32 = x.astype(np.complex64).astype(np.complex128)
    Wh, xh = _bf16(Dc), _bf16(x32)
    Wl, xl = _bf16(Dc - Wh), _bf16(x32 - xh)
    for v, hi, lo in ((Dc, Wh, Wl), (x32, xh, xl)):              # |v - hi - lo| <= 2^-16 |v| per real part
        assert np.all(np.abs((v - hi - lo).real) <= 2.0 ** -16 * np.abs(v.real))
        assert np.all(np.abs((v - hi - lo).imag) <= 2.0 ** -16 * np.abs(v.imag))
    ysp = ((Wh @ xh.reshape(-1)) + (Wl @ xh.reshape(-1)) + (Wh @ xl.reshape(-1))).reshape(Vc, ncd)
    assert np.all(np.abs(ysp - ref) <= U_SPLIT * B)
    assert _rel(ysp, ref) < REL_SPLIT
    for bad in ((Wh @ xh.reshape(-1)) + (Wh @ xl.reshape(-1)), (Wh @ xh.reshape(-1)) + (Wl @ xh.reshape(-1))):
        assert _rel(bad.reshape(Vc, ncd), ref) > 10 * REL_SPLIT
    ybad = ysp.copy()
    ybad[17] -= A[17, 3] @ x[nbr[17, 3]]
    assert np.any(np.abs(ybad - ref) > U_SPLIT * B)
