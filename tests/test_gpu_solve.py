"""Parity of the solver path: x = D^{-1} b from wd_solve against
dense LU (4^4 and a ragged small lattice) and, at larger size, against the
oracle's own operator on the returned x (true FP64 residual)."""
import numpy as np
import pytest

import synth
from oracle import solver, wilson
from tests.gpu_util import rel, to_dev

pytestmark = pytest.mark.gpu
BC = (1, 1, 1, -1)


@pytest.mark.parametrize("dims,kappa,spread", [((4, 4, 4, 4), 0.12, 0.3), ((2, 4, 6, 4), 0.13, 0.5)])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_solve_vs_dense(dims, kappa, spread, prec):
    from paper_2607_05157_b300 import Context
    U = synth.gauge_field(dims, spread, 1001)
    b = synth.spinors(dims, 3, 7)
    ctx = Context(dims, U, kappa, BC)
    x, it, res = ctx.solve(to_dev(b), tol=1e-10, prec=prec)
    x = x.cpu().numpy()
    D = wilson.sparse_matrix(U, kappa, BC).toarray()
    for r in range(3):
        xd = np.linalg.solve(D, b[r].reshape(-1))
        tr = np.linalg.norm(b[r].reshape(-1) - D @ x[r].reshape(-1)) / np.linalg.norm(b[r])
        assert tr <= 1e-10 * 1.01, tr
        assert abs(res[r] - tr) < 1e-11
        assert rel(x[r].reshape(-1), xd) < 1e-8
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_solve_8x8x8x16_true_residual(prec):
    """The 8^3 x 16 workload (kappa 0.125, spread 0.5): FP64 relative residual
    <= 1e-10 measured with the oracle's operator."""
    from paper_2607_05157_b300 import Context
    dims = (8, 8, 8, 16)
    U = synth.gauge_field(dims, 0.5, 1002)
    b = synth.spinors(dims, 4, 8)
    ctx = Context(dims, U, 0.125, BC)
    x, it, res = ctx.solve(to_dev(b), tol=1e-10, prec=prec)
    x = x.cpu().numpy()
    for r in range(4):
        tr = np.linalg.norm(b[r] - wilson.apply(U, x[r], 0.125, BC)) / np.linalg.norm(b[r])
        assert tr <= 1e-10 * 1.01, (r, tr, res[r], it[r])
    ctx.close()


def test_noconv_reported():
    from paper_2607_05157_b300 import Context, WD_ENOCONV
    dims = (4, 4, 4, 4)
    ctx = Context(dims, synth.gauge_field(dims, 0.3, 1), 0.12, BC)
    b = to_dev(synth.spinors(dims, 2, 1))
    x, it, res = ctx.solve(b, tol=1e-12, prec=1, max_iter=1, allow_noconv=True)
    assert np.all(res > 1e-12)
    import pytest as _p
    from paper_2607_05157_b300 import WDError
    with _p.raises(WDError) as e:
        ctx.solve(b, tol=1e-12, prec=1, max_iter=1)
    assert e.value.status == WD_ENOCONV
    ctx.close()


def test_zero_rhs():
    from paper_2607_05157_b300 import Context
    dims = (4, 4, 4, 4)
    ctx = Context(dims, synth.gauge_field(dims, 0.3, 1), 0.12, BC)
    b = np.zeros((2,) + synth.spinors(dims, 1, 0).shape[1:], np.complex128)
    b[1] = synth.spinors(dims, 1, 3)[0]
    x, it, res = ctx.solve(to_dev(b), tol=1e-10, prec=1)
    x = x.cpu().numpy()
    assert np.all(x[0] == 0) and res[0] == 0
    assert res[1] <= 1e-10
    ctx.close()


@pytest.mark.parametrize("prec", [1, 2])
def test_outer_double_float_vs_fp64(monkeypatch, prec):
    """Mixed solves whose FP64 steps use the double-float stencil (default)
    and the FP64 stencil (WD_DD=0): both meet 1e-10 by the oracle's own FP64
    residual, and their solutions agree to the tolerance."""
    from paper_2607_05157_b300 import Context
    dims = (8, 8, 8, 16)
    U = synth.gauge_field(dims, 0.5, 1002)
    b = synth.spinors(dims, 4, 41)
    xs = []
    for dd in ('1', '0'):
        monkeypatch.setenv('WD_DD', dd)
        ctx = Context(dims, U, 0.125, (1, 1, 1, -1))
        x, it, res = ctx.solve(to_dev(b), tol=1e-10, prec=prec)
        x = x.cpu().numpy()
        for r in range(4):
            rr = b[r] - wilson.apply(U, x[r], 0.125, (1, 1, 1, -1))
            assert np.linalg.norm(rr) <= 1e-10 * np.linalg.norm(b[r]) * 1.01
        xs.append(x)
        ctx.close()
    for r in range(4):
        assert rel(xs[0][r], xs[1][r]) < 1e-8


@pytest.mark.parametrize("variant", ["1", "11"])
def test_outer_double_float_variants(monkeypatch, variant):
    """Mixed FP32 solve with the scalar and the packed double-float stencil in
    the outer loop (the residual's odd intermediate in the double-float
    layout): 1e-10 by the oracle's FP64 residual."""
    from paper_2607_05157_b300 import Context
    monkeypatch.setenv('WD_DD_R', variant)
    dims = (4, 4, 6, 8)
    U = synth.gauge_field(dims, 0.5, 1006)
    b = synth.spinors(dims, 3, 43)
    ctx = Context(dims, U, 0.125, BC)
    x, it, res = ctx.solve(to_dev(b), tol=1e-10, prec=1)
    x = x.cpu().numpy()
    for r in range(3):
        rr = b[r] - wilson.apply(U, x[r], 0.125, BC)
        assert np.linalg.norm(rr) <= 1e-10 * np.linalg.norm(b[r]) * 1.01
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_graph_loop_matches_plain_loop(monkeypatch, prec):
    """The BiCGStab loop run as a captured CUDA graph with a device-side while
    node gives bit-identical solutions and iteration counts to the plain
    host-driven loop (the same kernels in the same order), on two solves in a
    row (the second replays the cached graph), and meets the tolerance.  The
    autotuner is off: it picks launch variants by timing, and variants that
    round differently would make the two contexts differ for that reason."""
    from paper_2607_05157_b300 import Context
    monkeypatch.setenv('WD_NO_AUTOTUNE', '1')
    dims = (4, 4, 6, 8)
    U = synth.gauge_field(dims, 0.5, 1007)
    b = synth.spinors(dims, 5, 44)
    out = {}
    for mode in ('graph', 'plain'):
        if mode == 'plain':
            monkeypatch.setenv('WD_NO_GRAPH', '1')
        ctx = Context(dims, U, 0.125, BC)
        runs = [ctx.solve(to_dev(b), tol=1e-10, prec=prec) for _ in range(2)]
        out[mode] = [(x.cpu().numpy(), it.copy()) for x, it, _ in runs]
        ctx.close()
    for (xg, ig), (xp, ip) in zip(out['graph'], out['plain']):
        assert np.array_equal(ig, ip)
        assert np.array_equal(xg, xp)
    x = out['graph'][1][0]
    for r in range(5):
        assert np.linalg.norm(b[r] - wilson.apply(U, x[r], 0.125, BC)) <= 1e-10 * np.linalg.norm(b[r]) * 1.01


@pytest.mark.parametrize("shift", [200, -200])
def test_fp64_norms_scale_invariant(shift):
    """The FP64 norms (squares summed on the FP32 pipes from an exact integer
    split of each double, with a running power-of-two exponent) keep the FP64
    solve invariant under scaling the source by 2^shift far outside the FP32
    range: the same iterations, the solution scaled bit for bit, the same
    reported residual.  The reported residual of a solve stopped early (so
    that the residual vector itself carries no cancellation) matches the
    oracle's FP64 residual of the returned solution to 1e-12 relative."""
    from paper_2607_05157_b300 import Context
    dims = (4, 4, 4, 8)
    U = synth.gauge_field(dims, 0.5, 1011)
    b = synth.spinors(dims, 3, 71)
    ctx = Context(dims, U, 0.125, BC)
    x1, it1, res1 = ctx.solve(to_dev(b), tol=1e-11, prec=0)
    x2, it2, res2 = ctx.solve(to_dev(b * 2.0 ** shift), tol=1e-11, prec=0)
    x3, _, res3 = ctx.solve(to_dev(b * 2.0 ** shift), tol=1e-11, prec=0, max_iter=3, allow_noconv=True)
    ctx.close()
    x1, x2, x3 = x1.cpu().numpy(), x2.cpu().numpy(), x3.cpu().numpy() / 2.0 ** shift
    assert np.array_equal(it1, it2)
    assert np.array_equal(x1 * 2.0 ** shift, x2)
    assert np.array_equal(res1, res2)
    assert np.all(res1 <= 1e-11)
    D = wilson.sparse_matrix(U, 0.125, BC)
    for r in range(3):
        tr = np.linalg.norm(b[r].reshape(-1) - D @ x3[r].reshape(-1)) / np.linalg.norm(b[r])
        assert tr > 1e-5
        assert abs(res3[r] - tr) <= 1e-12 * tr


@pytest.mark.parametrize("shift", [40, -40, 200, -200, 133, -134])
def test_mixed_solve_scale_invariant(shift):
    """The mixed-precision solve is invariant under scaling the source by
    2^shift: the outer residual (double-float layout), its norm (running
    power-of-two exponent) and its scaled FP32 copy (scale applied as a power
    of two and an FP32 significand) all commute with the scaling, the inner
    FP32 solves see the same normalised residuals, and a source whose norm
    leaves [2^-30, 2^30] (2^+-200, 1e+-40: outside the double-float range) is
    solved at a power-of-two scale of norm in [1, 2) -- the same iterations,
    the solution scaled bit for bit, the same reported residual."""
    from paper_2607_05157_b300 import Context
    dims = (4, 4, 4, 8)
    U = synth.gauge_field(dims, 0.5, 1012)
    b = synth.spinors(dims, 3, 72)
    ctx = Context(dims, U, 0.125, BC)
    x1, it1, res1 = ctx.solve(to_dev(b), tol=1e-10, prec=1)
    x2, it2, res2 = ctx.solve(to_dev(b * 2.0 ** shift), tol=1e-10, prec=1)
    ctx.close()
    x1, x2 = x1.cpu().numpy(), x2.cpu().numpy()
    assert np.array_equal(it1, it2)
    assert np.array_equal(x1 * 2.0 ** shift, x2)
    assert np.array_equal(res1, res2)
    D = wilson.sparse_matrix(U, 0.125, BC)
    for r in range(3):
        tr = np.linalg.norm(b[r].reshape(-1) - D @ x1[r].reshape(-1)) / np.linalg.norm(b[r])
        assert tr <= 1e-10 * 1.01
