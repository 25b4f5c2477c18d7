"""Parity of the point-source pseudoscalar correlator (the 8^3 x 16 workload's
C(t) from 12 point sources): the free field at full size against the
momentum-sum closed form, and an interacting 4^4 field against dense LU."""
import numpy as np
import pytest

import synth
from oracle import freefield, solver, wilson

pytestmark = pytest.mark.gpu
BC = (1, 1, 1, -1)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_free_field_8x8x8x16(prec):
    from paper_2607_05157_b300 import Context, wd_point_correlator
    dims = (8, 8, 8, 16)
    ctx = Context(dims, synth.unit_gauge(dims), 0.125, BC)
    C = wd_point_correlator(ctx.h, (0, 0, 0, 0), dims[3], prec=prec, tol=1e-12)
    ref = freefield.pion_correlator(dims, 0.125, BC)
    assert np.abs(C - ref).max() <= 1e-9 * np.abs(ref).max()
    ctx.close()


def test_interacting_dense_4x4x4x4():
    from paper_2607_05157_b300 import Context, wd_point_correlator
    dims, kappa = (4, 4, 4, 4), 0.12
    U = synth.gauge_field(dims, 0.3, 1001)
    ctx = Context(dims, U, kappa, BC)
    src = (1, 2, 3, 2)
    C = wd_point_correlator(ctx.h, src, dims[3], prec=1, tol=1e-12)
    Dinv = solver.dense_inverse(wilson.sparse_matrix(U, kappa, BC))
    site0 = wilson.site_index(dims, *src)
    cols = Dinv[:, 12 * site0:12 * site0 + 12]
    ref = (np.abs(cols) ** 2).reshape(dims[3], -1).sum(axis=1)
    assert np.abs(C - ref).max() <= 1e-9 * ref.max()
    ctx.close()
