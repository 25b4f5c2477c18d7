"""Parity of every stencil launch variant of the fine stencil (plain, software-pipelined,
timeslices staged through shared memory by bulk async copies, register-capped
with grouped RHS block orders) with the oracle,
each forced through the launch-shape override, FP32 and BF16, D and D^dag, with
a ragged RHS count, plus a mixed-precision solve on the staged variant."""
import os

import numpy as np
import pytest

import synth
from oracle import wilson
from tests.gpu_util import rel, to_dev
from tests.test_gpu_dslash import ELEM_U, abs_stencil_bound, assert_elementwise

pytestmark = pytest.mark.gpu
BC = (1, 1, 1, -1)


@pytest.fixture
def override():
    def set_r(r):
        os.environ['WD_HOP_R'] = str(r)
    yield set_r
    os.environ.pop('WD_HOP_R', None)


@pytest.mark.parametrize("code", [1, 2, 4, 11, 12, 21, 22, 24, 31, 32, 41, 42, 51, 52, 54, 62, 63, 64, "65:32", "63:128"])
@pytest.mark.parametrize("prec,tol", [(1, 3e-6), (2, 2e-2)])
@pytest.mark.parametrize("dagger", [False, True])
def test_variant_parity(override, code, prec, tol, dagger):
    import torch
    from paper_2607_05157_b300 import Context
    override(code)
    dims = (8, 8, 8, 16)            # timeslice of 256 half-sites: the staged variant applies
    U = synth.gauge_field(dims, 0.5, 1002)
    psi = synth.spinors(dims, 7, 33).astype(np.complex64).astype(np.complex128)
    ctx = Context(dims, U, 0.125, BC)
    y = ctx.apply(to_dev(psi, torch.complex64), prec=prec, dagger=dagger).cpu().numpy()
    f = wilson.apply_dagger if dagger else wilson.apply
    for r in (0, 3, 6):
        ref = f(U, psi[r], 0.125, BC)
        assert rel(y[r], ref) < tol
        assert_elementwise(y[r], ref, abs_stencil_bound(U, psi[r], 0.125), ELEM_U[prec], (code, r))
    ctx.close()


@pytest.mark.parametrize("code", [21, 22])
def test_staged_solve(override, code):
    from paper_2607_05157_b300 import Context
    override(code)
    dims = (8, 8, 8, 16)
    U = synth.gauge_field(dims, 0.5, 1002)
    b = synth.spinors(dims, 5, 8)
    ctx = Context(dims, U, 0.125, BC)
    x, it, res = ctx.solve(to_dev(b), tol=1e-10, prec=1)
    x = x.cpu().numpy()
    for r in range(5):
        tr = np.linalg.norm(b[r] - wilson.apply(U, x[r], 0.125, BC)) / np.linalg.norm(b[r])
        assert tr <= 1e-10 * 1.01
    ctx.close()


@pytest.mark.parametrize("dims", [(8, 8, 8, 16), (4, 6, 8, 10), (6, 4, 4, 6)])
@pytest.mark.parametrize("nrhs", [1, 5])
@pytest.mark.parametrize("dagger", [False, True])
def test_plane_walk_parity(override, dims, nrhs, dagger):
    """The plane-walk variant (code 71: persistent CTAs walking z with a ring
    of x-y planes in shared memory, one thread per site and RHS) against the
    oracle, element by element, on non-cubic lattices (plane neighbours in x
    and y, the z ring and the t neighbours all wrap), with a ragged RHS
    tile."""
    import torch
    from paper_2607_05157_b300 import Context
    override(71)
    U = synth.gauge_field(dims, 0.5, 1006)
    psi = synth.spinors(dims, nrhs, 34).astype(np.complex64).astype(np.complex128)
    ctx = Context(dims, U, 0.125, BC)
    y = ctx.apply(to_dev(psi, torch.complex64), prec=1, dagger=dagger).cpu().numpy()
    f = wilson.apply_dagger if dagger else wilson.apply
    for r in range(nrhs):
        ref = f(U, psi[r], 0.125, BC)
        assert rel(y[r], ref) < 3e-6
        assert_elementwise(y[r], ref, abs_stencil_bound(U, psi[r], 0.125), ELEM_U[1], (dims, r))
    ctx.close()


def test_plane_walk_solve(override):
    """A mixed-precision solve on the plane-walk variant: its launches walk
    the list of RHS still converging (inside the CUDA-graph loop)."""
    from paper_2607_05157_b300 import Context
    override(71)
    dims = (8, 8, 8, 16)
    U = synth.gauge_field(dims, 0.5, 1002)
    b = synth.spinors(dims, 5, 8)
    b[3] *= 1e-3                                    # converges at its own pace
    ctx = Context(dims, U, 0.125, BC)
    x, it, res = ctx.solve(to_dev(b), tol=1e-10, prec=1)
    x = x.cpu().numpy()
    for r in range(5):
        tr = np.linalg.norm(b[r] - wilson.apply(U, x[r], 0.125, BC)) / np.linalg.norm(b[r])
        assert tr <= 1e-10 * 1.01
    ctx.close()
