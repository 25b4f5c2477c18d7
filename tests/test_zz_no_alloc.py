"""wd_apply_noalloc: the allocation-free variant of wd_apply, for callers that
cannot allocate device memory while running (fixed device-memory budgets,
frameworks whose caching allocator must own all device memory).  Called through
the C ABI and compared with wd_apply on two calls in a row; this file sorts
last so that a run stopping at the first failure has run every other test."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
BC = (1, 1, 1, -1)


def _call(fn, ctx, x, out, prec, dagger):
    return fn(ctx.h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), x.shape[0], prec, dagger)


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 3e-6), (2, 1e-2)])
def test_noalloc_matches_apply_twice(prec, tol):
    import torch
    from paper_2607_05157_b300 import Context, lib, WD_OK
    dims = (8, 8, 8, 16)
    U = synth.gauge_field(dims, 0.5, 1002)
    ctx = Context(dims, U, 0.125, BC)
    dt = torch.complex128 if prec == 0 else torch.complex64
    for call, (nrhs, dagger) in enumerate([(3, 0), (5, 1)]):
        x = torch.from_numpy(synth.spinors(dims, nrhs, 40 + call)).to(dt).cuda()
        ref = torch.empty_like(x)
        got = torch.full_like(x, float('nan'))
        assert _call(lib.wd_apply, ctx, x, ref, prec, dagger) == WD_OK
        # a first call loads the kernels it uses (code, not data); the second one
        # is checked to leave the device's free memory as it was: nothing allocated
        assert _call(lib.wd_apply_noalloc, ctx, x, got, prec, dagger) == WD_OK
        got.fill_(float('nan'))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        assert _call(lib.wd_apply_noalloc, ctx, x, got, prec, dagger) == WD_OK
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        a, b = got.cpu().numpy(), ref.cpu().numpy()
        for r in range(nrhs):
            assert np.linalg.norm(a[r] - b[r]) <= tol * np.linalg.norm(b[r])
    ctx.close()


def test_noalloc_rejects_oversize():
    import torch
    from paper_2607_05157_b300 import Context, lib
    from paper_2607_05157_b300._lib import WD_EINVAL
    dims = (16, 16, 16, 32)                       # FP64: 384 B x 131072 sites = 48 MiB per RHS
    ctx = Context(dims, synth.gauge_field(dims, 0.5, 1), 0.13, BC)
    x = torch.zeros(ctx.field_shape(2), dtype=torch.complex128, device='cuda')
    out = torch.empty_like(x)
    assert _call(lib.wd_apply_noalloc, ctx, x, out, 0, 0) == WD_EINVAL
    assert b'static scratch' in lib.wd_last_error()
    ctx.close()
