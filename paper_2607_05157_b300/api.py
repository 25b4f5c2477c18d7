"""Python binding: the C ABI of include/wd.h with the same names.

Argument marshalling only -- torch CUDA tensors are passed as device
pointers, numpy arrays as host pointers; every computation happens in
libwd.so on the GPU.
"""
import ctypes

import numpy as np

from ._lib import lib, check, WD_OK, WD_ENOCONV, WD_EBREAKDOWN, WD_FP64, WD_MIXED_FP32, WD_FP64_DD, WDError

_ci = ctypes.c_int


def _iarr(vals):
    vals = [int(v) for v in vals]
    return (_ci * len(vals))(*vals)


def _dev_ptr(t, dtype=None, name='tensor'):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f'{name} must be a CUDA tensor')
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f'{name} must have dtype {dtype}, got {t.dtype}')
    if not t.is_contiguous():
        raise ValueError(f'{name} must be contiguous')
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def wd_create(dims, gauge, kappa, bc, stream=None):
    g = np.ascontiguousarray(gauge, dtype=np.complex128)
    X, Y, Z, T = dims
    if g.shape != (4, T, Z, Y, X, 3, 3):
        raise ValueError(f'gauge must have shape (4, T, Z, Y, X, 3, 3), got {g.shape}')
    h = ctypes.c_void_p()
    check(lib.wd_create(ctypes.byref(h), _iarr(dims), _host_ptr(g), float(kappa), _iarr(bc), _stream_ptr(stream)),
          'wd_create')
    return h


def wd_destroy(h):
    check(lib.wd_destroy(h), 'wd_destroy')


def wd_update_gauge(h, gauge, kappa):
    g = np.ascontiguousarray(gauge, dtype=np.complex128)
    check(lib.wd_update_gauge(h, _host_ptr(g), float(kappa)), 'wd_update_gauge')


def wd_apply(h, x, out, prec=WD_FP64, dagger=False):
    import torch
    dt = torch.complex128 if prec in (WD_FP64, WD_FP64_DD) else torch.complex64
    check(lib.wd_apply(h, _dev_ptr(x, dt, 'in'), _dev_ptr(out, dt, 'out'), x.shape[0], int(prec), int(bool(dagger))),
          'wd_apply')
    return out


def wd_solve(h, b, x, tol, prec=WD_MIXED_FP32, max_iter=10000, allow_noconv=False):
    """Returns (status, iters[nrhs], true_resid[nrhs])."""
    import torch
    n = b.shape[0]
    iters = np.zeros(n, np.int32)
    res = np.zeros(n, np.float64)
    s = lib.wd_solve(h, _dev_ptr(b, torch.complex128, 'rhs'), _dev_ptr(x, torch.complex128, 'x'), n, float(tol),
                     int(prec), int(max_iter), _host_ptr(iters), _host_ptr(res))
    if s != WD_OK and not (allow_noconv and s in (WD_ENOCONV, WD_EBREAKDOWN)):
        check(s, 'wd_solve')
    return s, iters, res


def probe_color(dims, d, with_colors=True):
    """Returns (n_c, sigma tuple, colours or None)."""
    nD = len(dims)
    nc = _ci()
    sig = (_ci * nD)()
    cols = np.zeros(int(np.prod(dims)), np.int32) if with_colors else None
    check(lib.probe_color(_iarr(dims), nD, int(d), ctypes.byref(nc), sig,
                          _host_ptr(cols) if with_colors else None), 'probe_color')
    return nc.value, tuple(sig[j] for j in range(nD)), cols


def trace_estimate(h, method, dilution, N, T, n2=0, d=0, seed=0, op=1, prec=WD_MIXED_FP32, batch=0, tol=1e-10,
                   with_samples=False):
    """Returns dict(estimate (T,) complex, total complex, var (T,), var_total, n_solves, samples (N, T) or None)."""
    est = np.zeros(2 * (T + 1), np.float64)
    var = np.zeros(T + 1, np.float64)
    ns = ctypes.c_int64()
    smp = np.zeros((N, T, 2), np.float64) if with_samples else None
    check(lib.trace_estimate(h, int(method), int(dilution), int(N), int(n2), int(d), ctypes.c_uint64(seed), int(op),
                             int(prec), int(batch), float(tol), _host_ptr(est), _host_ptr(var), ctypes.byref(ns),
                             _host_ptr(smp) if with_samples else None), 'trace_estimate')
    e = est[0::2] + 1j * est[1::2]
    out = dict(estimate=e[:T], total=e[T], var=var[:T], var_total=var[T], n_solves=ns.value, samples=None)
    if with_samples:
        out['samples'] = smp[..., 0] + 1j * smp[..., 1]
    return out


def wd_point_correlator(h, src, T, prec=WD_MIXED_FP32, tol=1e-10):
    """C(t) (numpy, length T) from 12 point sources at site src = (x, y, z, t)."""
    C = np.zeros(T, np.float64)
    check(lib.wd_point_correlator(h, _iarr(src), int(prec), float(tol), _host_ptr(C)), 'wd_point_correlator')
    return C


def wd_connected_mlmc(h, N1, N2, T, seed=0, prec=WD_MIXED_FP32, tol=1e-10, batch=0, with_samples=False):
    """Connected G(t) with the two-level decomposition.  Returns dict(G (6, T)
    complex: (1,1), (1,2), (2,1), (2,2), total, plain; var (6, T);
    samples1 (N1, 4, T) and samples2 (N2, T) or None; n_solves)."""
    G = np.zeros((6, T, 2), np.float64)
    var = np.zeros((6, T), np.float64)
    s1 = np.zeros((N1, 4, T, 2), np.float64) if with_samples else None
    s2 = np.zeros((N2, T, 2), np.float64) if with_samples else None
    ns = ctypes.c_int64()
    check(lib.wd_connected_mlmc(h, int(N1), int(N2), ctypes.c_uint64(seed), int(prec), float(tol), int(batch),
                                _host_ptr(G), _host_ptr(var), _host_ptr(s1) if with_samples else None,
                                _host_ptr(s2) if with_samples else None, ctypes.byref(ns)), 'wd_connected_mlmc')
    out = dict(G=G[..., 0] + 1j * G[..., 1], var=var, n_solves=ns.value, samples1=None, samples2=None)
    if with_samples:
        out['samples1'] = s1[..., 0] + 1j * s1[..., 1]
        out['samples2'] = s2[..., 0] + 1j * s2[..., 1]
    return out


def trace_estimate_mlmc_probe(h, dilution, d, N1, coarse_dil, d2, N2, T, seed=0, op=1, prec=WD_MIXED_FP32, batch=0,
                              tol=1e-10):
    """Two-level MLMC with probing on both levels.  Returns dict(estimate (T,),
    total, var (T,), var_total, n_solves, samples1 (N1, T), samples2 (N2, T))."""
    est = np.zeros(2 * (T + 1), np.float64)
    var = np.zeros(T + 1, np.float64)
    ns = ctypes.c_int64()
    s1 = np.zeros((N1, T, 2), np.float64)
    s2 = np.zeros((N2, T, 2), np.float64)
    check(lib.trace_estimate_mlmc_probe(h, int(dilution), int(d), int(N1), int(coarse_dil), int(d2), int(N2),
                                        ctypes.c_uint64(seed), int(op), int(prec), int(batch), float(tol),
                                        _host_ptr(est), _host_ptr(var), ctypes.byref(ns), _host_ptr(s1),
                                        _host_ptr(s2)), 'trace_estimate_mlmc_probe')
    e = est[0::2] + 1j * est[1::2]
    return dict(estimate=e[:T], total=e[T], var=var[:T], var_total=var[T], n_solves=ns.value,
                samples1=s1[..., 0] + 1j * s1[..., 1], samples2=s2[..., 0] + 1j * s2[..., 1])


def wd_mg3_setup(h, tv2, nv2, agg2, tv_iters=3, seed=0):
    ptr = None
    if tv2 is not None:
        tv2 = np.ascontiguousarray(tv2, dtype=np.complex128)
        ptr = _host_ptr(tv2)
    check(lib.wd_mg3_setup(h, ptr, int(nv2), _iarr(agg2), int(tv_iters), ctypes.c_uint64(seed)), 'wd_mg3_setup')


def wd_coarse3_apply(h, x, out):
    import torch
    check(lib.wd_coarse3_apply(h, _dev_ptr(x, torch.complex128, 'in'), _dev_ptr(out, torch.complex128, 'out'),
                               x.shape[0]), 'wd_coarse3_apply')
    return out


def wd_restrict2(h, y2, y3):
    import torch
    check(lib.wd_restrict2(h, _dev_ptr(y2, torch.complex128), _dev_ptr(y3, torch.complex128), y2.shape[0]),
          'wd_restrict2')
    return y3


def wd_prolong2(h, y3, y2):
    import torch
    check(lib.wd_prolong2(h, _dev_ptr(y3, torch.complex128), _dev_ptr(y2, torch.complex128), y3.shape[0]),
          'wd_prolong2')
    return y2


def trace_estimate_mlmc3(h, N1, N2, N3, T, seed=0, op=1, prec=WD_MIXED_FP32, batch=0, tol=1e-10):
    """Three-level MLMC.  Returns dict(estimate (T,), total, var (T,), var_total,
    n_solves, samples1 (N1, T), samples2 (N2, T), samples3 (N3, T))."""
    est = np.zeros(2 * (T + 1), np.float64)
    var = np.zeros(T + 1, np.float64)
    ns = ctypes.c_int64()
    S = [np.zeros((N, T, 2), np.float64) for N in (N1, N2, N3)]
    check(lib.trace_estimate_mlmc3(h, int(N1), int(N2), int(N3), ctypes.c_uint64(seed), int(op), int(prec),
                                   int(batch), float(tol), _host_ptr(est), _host_ptr(var), ctypes.byref(ns),
                                   _host_ptr(S[0]), _host_ptr(S[1]), _host_ptr(S[2])), 'trace_estimate_mlmc3')
    e = est[0::2] + 1j * est[1::2]
    out = dict(estimate=e[:T], total=e[T], var=var[:T], var_total=var[T], n_solves=ns.value)
    for l in range(3):
        out['samples%d' % (l + 1)] = S[l][..., 0] + 1j * S[l][..., 1]
    return out


def mlmc_allocate(V, C, eps):
    """Samples per level (int64 array) for variances V, costs C and a target
    standard error eps (host computation in libwd)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    C = np.ascontiguousarray(C, dtype=np.float64)
    if V.shape != C.shape or V.ndim != 1:
        raise ValueError('V and C must be 1-D arrays of the same length')
    N = np.zeros(V.shape[0], np.int64)
    check(lib.mlmc_allocate(int(V.shape[0]), _host_ptr(V), _host_ptr(C), float(eps), _host_ptr(N)), 'mlmc_allocate')
    return N


def wd_mlmc_level2_samples(h, n2, T):
    smp = np.zeros((n2, T, 2), np.float64)
    check(lib.wd_mlmc_level2_samples(h, _host_ptr(smp), int(n2)), 'wd_mlmc_level2_samples')
    return smp[..., 0] + 1j * smp[..., 1]


def wd_mg_setup(h, tv, nv, agg, tv_iters=3, seed=0):
    ptr = None
    if tv is not None:
        tv = np.ascontiguousarray(tv, dtype=np.complex128)
        ptr = _host_ptr(tv)
    check(lib.wd_mg_setup(h, ptr, int(nv), _iarr(agg), int(tv_iters), ctypes.c_uint64(seed)), 'wd_mg_setup')


def wd_mg_test_vectors(h, nv, iters, seed, out):
    import torch
    check(lib.wd_mg_test_vectors(h, int(nv), int(iters), ctypes.c_uint64(seed), _dev_ptr(out, torch.complex128, 'out')),
          'wd_mg_test_vectors')
    return out


def wd_coarse_apply(h, x, out, prec=WD_FP64):
    import torch
    check(lib.wd_coarse_apply(h, _dev_ptr(x, torch.complex128, 'in'), _dev_ptr(out, torch.complex128, 'out'),
                              x.shape[0], int(prec)), 'wd_coarse_apply')
    return out


def wd_restrict(h, fine, coarse):
    import torch
    check(lib.wd_restrict(h, _dev_ptr(fine, torch.complex128), _dev_ptr(coarse, torch.complex128), fine.shape[0]),
          'wd_restrict')
    return coarse


def wd_prolong(h, coarse, fine):
    import torch
    check(lib.wd_prolong(h, _dev_ptr(coarse, torch.complex128), _dev_ptr(fine, torch.complex128), coarse.shape[0]),
          'wd_prolong')
    return fine


def wd_coarse_solve(h, b, x, tol, prec=WD_MIXED_FP32, max_iter=10000):
    import torch
    n = b.shape[0]
    res = np.zeros(n, np.float64)
    check(lib.wd_coarse_solve(h, _dev_ptr(b, torch.complex128), _dev_ptr(x, torch.complex128), n, float(tol),
                              int(prec), int(max_iter), _host_ptr(res)), 'wd_coarse_solve')
    return res


def wd_link_force(h, w, z, G, H, accumulate=False):
    import torch
    check(lib.wd_link_force(h, _dev_ptr(w, torch.complex128, 'w'), _dev_ptr(z, torch.complex128, 'z'), w.shape[0],
                            _dev_ptr(G, torch.complex128, 'G'), _dev_ptr(H, torch.complex128, 'H'),
                            int(bool(accumulate))), 'wd_link_force')


def wd_profile(h, enable):
    check(lib.wd_profile(h, int(bool(enable))), 'wd_profile')


def wd_profile_get(h, kernel):
    n = ctypes.c_int64()
    ms = ctypes.c_double()
    by = ctypes.c_double()
    check(lib.wd_profile_get(h, int(kernel), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)), 'wd_profile_get')
    return n.value, ms.value, by.value


def wd_launch_count(h):
    return int(lib.wd_launch_count(h))


class Context:
    """Owns one wd_ctx: a gauge field on one lattice with kappa and bc."""

    def __init__(self, dims, gauge, kappa, bc=(1, 1, 1, -1), stream=None):
        self.dims = tuple(int(v) for v in dims)
        self.kappa = float(kappa)
        self.bc = tuple(int(v) for v in bc)
        self.h = wd_create(self.dims, gauge, kappa, bc, stream)

    @property
    def T(self):
        return self.dims[3]

    def field_shape(self, nrhs):
        X, Y, Z, T = self.dims
        return (nrhs, T, Z, Y, X, 4, 3)

    def apply(self, x, prec=WD_FP64, dagger=False):
        import torch
        out = torch.empty_like(x)
        return wd_apply(self.h, x, out, prec, dagger)

    def solve(self, b, tol=1e-10, prec=WD_MIXED_FP32, max_iter=10000, allow_noconv=False):
        import torch
        x = torch.empty_like(b)
        s, it, res = wd_solve(self.h, b, x, tol, prec, max_iter, allow_noconv)
        return x, it, res

    def close(self):
        if getattr(self, 'h', None) is not None:
            wd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trace_gradient(h, method, dilution, N, T, d=0, seed=0, op=1, prec=WD_MIXED_FP32, batch=0, tol=1e-10,
                   weights=None, G=None, H=None, link_shape=None):
    """Returns (dkappa, G, H) for L = Re sum_t weights[t] mean_i X_i(t)."""
    import torch
    if G is None:
        G = torch.empty(link_shape, dtype=torch.complex128, device='cuda')
        H = torch.empty_like(G)
    w = None
    if weights is not None:
        w = np.ascontiguousarray(weights, dtype=np.float64)
        assert w.shape == (T,)
    dk = ctypes.c_double()
    check(lib.trace_gradient(h, int(method), int(dilution), int(N), int(d), ctypes.c_uint64(seed), int(op),
                             int(prec), int(batch), float(tol), _host_ptr(w) if w is not None else None,
                             ctypes.byref(dk), _dev_ptr(G, torch.complex128, 'G'), _dev_ptr(H, torch.complex128, 'H')),
          'trace_gradient')
    return dk.value, G, H


class Batch:
    """wd_batch over several Contexts sharing one stream (lattices of any sizes)."""

    def __init__(self, contexts):
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c.h.value for c in self.contexts])
        self.h = ctypes.c_void_p()
        check(lib.wd_batch_create(ctypes.byref(self.h), arr, len(self.contexts)), 'wd_batch_create')

    def solve(self, rhs, tol=1e-10, prec=WD_MIXED_FP32, max_iter=100000, use_graph=True):
        """rhs: list of complex128 CUDA tensors; returns (xs, iters[n], resid[sum nrhs])."""
        import torch
        xs = [torch.empty_like(b) for b in rhs]
        n = len(rhs)
        rp = (ctypes.c_void_p * n)(*[_dev_ptr(b, torch.complex128).value for b in rhs])
        xp = (ctypes.c_void_p * n)(*[_dev_ptr(x, torch.complex128).value for x in xs])
        nr = (ctypes.c_int * n)(*[b.shape[0] for b in rhs])
        iters = np.zeros(n, np.int32)
        res = np.zeros(sum(b.shape[0] for b in rhs), np.float64)
        check(lib.wd_batch_solve(self.h, rp, xp, nr, float(tol), int(prec), int(max_iter), int(bool(use_graph)),
                                 _host_ptr(iters), _host_ptr(res)), 'wd_batch_solve')
        return xs, iters, res

    def close(self):
        if getattr(self, 'h', None) is not None:
            lib.wd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
