"""ctypes declarations of the C ABI in include/wd.h (no computation here)."""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, 'libwd.so')

WD_OK, WD_EINVAL, WD_ENOMEM, WD_ECUDA, WD_ENOCONV, WD_EBREAKDOWN, WD_ETIMEOUT, WD_ENOTSUP = 0, -1, -2, -3, -4, -5, -6, -7
WD_FP64, WD_MIXED_FP32, WD_MIXED_BF16, WD_FP64_DD = 0, 1, 2, 3
WD_HUTCH, WD_PROBE, WD_MLMC2, WD_MLMC2_PROBE = 0, 1, 2, 3
WD_TR_DINV, WD_TR_G5_DINV = 0, 1
WD_DIL_TIME, WD_COLOR_3D = 0x100, 0x200
WD_K_HOP, WD_K_BLAS, WD_K_COARSE, WD_K_FORCE, WD_K_HOP64, WD_K_COUNT = 0, 1, 2, 3, 4, 5

_NAMES = {0: 'WD_OK', -1: 'WD_EINVAL', -2: 'WD_ENOMEM', -3: 'WD_ECUDA', -4: 'WD_ENOCONV',
          -5: 'WD_EBREAKDOWN', -6: 'WD_ETIMEOUT', -7: 'WD_ENOTSUP'}


class WDError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f'{where}: {_NAMES.get(status, status)}: {msg}')
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f'libwd.so not built ({LIB_PATH}); run python paper_2607_05157_b300/build.py')

lib = ctypes.CDLL(LIB_PATH)

c_int, c_double, c_void_p, c_int64, c_uint64 = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64
P = ctypes.POINTER

_SIGS = {
    'wd_create': (c_int, [P(c_void_p), P(c_int), c_void_p, c_double, P(c_int), c_void_p]),
    'wd_destroy': (c_int, [c_void_p]),
    'wd_apply': (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int]),
    'wd_apply_noalloc': (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int]),
    'wd_batch_create': (c_int, [P(c_void_p), P(c_void_p), c_int]),
    'wd_batch_destroy': (c_int, [c_void_p]),
    'wd_batch_solve': (c_int, [c_void_p, P(c_void_p), P(c_void_p), P(c_int), c_double, c_int, c_int, c_int,
                               c_void_p, c_void_p]),
    'wd_solve': (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, c_int, c_int, c_void_p, c_void_p]),
    'probe_color': (c_int, [P(c_int), c_int, c_int, P(c_int), P(c_int), c_void_p]),
    'trace_estimate': (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_uint64, c_int, c_int, c_int,
                               c_double, c_void_p, c_void_p, P(c_int64), c_void_p]),
    'wd_mlmc_level2_samples': (c_int, [c_void_p, c_void_p, c_int]),
    'mlmc_allocate': (c_int, [c_int, c_void_p, c_void_p, c_double, c_void_p]),
    'wd_mg3_setup': (c_int, [c_void_p, c_void_p, c_int, P(c_int), c_int, c_uint64]),
    'wd_coarse3_apply': (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    'wd_restrict2': (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    'wd_prolong2': (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    'trace_estimate_mlmc3': (c_int, [c_void_p, c_int, c_int, c_int, c_uint64, c_int, c_int, c_int, c_double, c_void_p,
                                     c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    'trace_estimate_mlmc_probe': (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_int, c_uint64, c_int, c_int,
                                          c_int, c_double, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    'wd_connected_mlmc': (c_int, [c_void_p, c_int, c_int, c_uint64, c_int, c_double, c_int, c_void_p, c_void_p,
                                  c_void_p, c_void_p, c_void_p]),
    'wd_point_correlator': (c_int, [c_void_p, P(c_int), c_int, c_double, c_void_p]),
    'wd_last_error': (ctypes.c_char_p, []),
    'wd_mg_setup': (c_int, [c_void_p, c_void_p, c_int, P(c_int), c_int, c_uint64]),
    'wd_mg_test_vectors': (c_int, [c_void_p, c_int, c_int, c_uint64, c_void_p]),
    'wd_coarse_apply': (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int]),
    'wd_restrict': (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    'wd_prolong': (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    'wd_coarse_solve': (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, c_int, c_int, c_void_p]),
    'wd_link_force': (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_int]),
    'wd_update_gauge': (c_int, [c_void_p, c_void_p, c_double]),
    'trace_gradient': (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_uint64, c_int, c_int, c_int, c_double,
                               c_void_p, P(c_double), c_void_p, c_void_p]),
    'wd_profile': (c_int, [c_void_p, c_int]),
    'wd_profile_get': (c_int, [c_void_p, c_int, P(c_int64), P(c_double), P(c_double)]),
    'wd_launch_count': (c_int64, [c_void_p]),
}

for _n, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _n)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


def check(status, where):
    if status != WD_OK:
        raise WDError(status, where, lib.wd_last_error().decode(errors='replace'))
    return status
