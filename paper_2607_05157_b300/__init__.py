"""B300-native engine for the hot path of stochastic trace estimation with the
Wilson-Dirac operator (Hutchinson, torus-colouring probing x dilution, two-level
multigrid MLMC), after "Variance reduction with probing and Multilevel Monte
Carlo in Lattice QCD".

Every computation runs in libwd.so (hand-written sm_103a CUDA behind the C ABI
of include/wd.h).  This package is the thin Python binding: the functions here
carry the C names and only marshal arguments (torch tensors -> device pointers,
numpy arrays -> host pointers).  There is no CPU fallback: importing the
package fails if libwd.so is missing, and every call raises WDError on a
non-zero status.
"""
from ._lib import (WDError, lib, WD_OK, WD_ENOCONV, WD_EBREAKDOWN, WD_FP64, WD_MIXED_FP32, WD_MIXED_BF16, WD_FP64_DD,
                   WD_HUTCH, WD_PROBE, WD_MLMC2, WD_MLMC2_PROBE, WD_TR_DINV, WD_TR_G5_DINV, WD_DIL_TIME, WD_COLOR_3D,
                   WD_K_HOP, WD_K_BLAS, WD_K_COARSE, WD_K_FORCE, WD_K_HOP64)
from .api import (Context, Batch, wd_create, wd_destroy, wd_apply, wd_solve, probe_color, trace_estimate,
                  wd_mg_setup, wd_mg_test_vectors, wd_coarse_apply, wd_restrict, wd_prolong, wd_coarse_solve, wd_link_force,
                  wd_update_gauge, wd_profile, wd_profile_get, wd_launch_count, wd_mlmc_level2_samples,
                  trace_gradient, wd_point_correlator, mlmc_allocate, wd_connected_mlmc, trace_estimate_mlmc_probe,
                  wd_mg3_setup, wd_coarse3_apply, wd_restrict2, wd_prolong2, trace_estimate_mlmc3)

__all__ = [n for n in dir() if not n.startswith('_')]
