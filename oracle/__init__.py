"""FP64 CPU oracle for the Wilson-Dirac trace-estimation hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, call, link or execute anything in this
package; only the test-suite, the smoke check and the benchmark's CPU-baseline
leg use it.  It shares no code with the CUDA path: the noise hash, the
colouring search, the stencil and every estimator are written here
independently, from the paper's definitions, in plain numpy/scipy (and plain
C for the integer colouring search).

Modules
  gamma       -- Euclidean chiral gamma matrices (Sec. 1 states only "spin 4 x
                 colour 3"; the basis is a documented reading).
  wilson      -- the Wilson-Dirac operator D (Sec. 1: 12x12 blocks on a 4D
                 nearest-neighbour torus), as a vectorised stencil and as an
                 explicitly assembled sparse matrix.
  noise       -- Rademacher vectors (Sec. 1) from a splitmix64 counter hash.
  coloring    -- torus colouring c(x) = sum_j sigma_j x_j mod n_c (Sec. 3,
                 Eq. 15) and its exhaustive search (Sec. 3, Table 1).
  solver      -- FP64 BiCGStab and dense LU (the D^{-1} eta products of Sec. 1).
  freefield   -- closed-form free-field (U = 1) propagator by momentum sums.
  estimators  -- Hutchinson (Eq. 3), probing x dilution (Eqs. 13-14, Sec. 3),
                 two-level multigrid MLMC (Eqs. 9-12) and exact variances (Eq. 4).
  multigrid   -- aggregation prolongator P (P^dagger P = I) and Galerkin
                 coarse operator D_c = P^dagger D P (Sec. 2, Eq. 7).
  gradient    -- dense derivative -tr(B D^{-1} dD D^{-1}) and the per-link
                 force contraction.

Equations are numbered in order of appearance in the paper (Eq. 1 = the
noise moments, Eq. 3 = the Hutchinson estimator, Eq. 4 = its variance,
Eq. 7 = Galerkin, Eq. 15 = the colouring formula, Eq. 21 = O(t)).

Parity unpinned: nothing.  Every function is checked in tests/ against a
closed form, an invariant, a brute-force enumeration or a value the paper
prints (see tests/test_oracle_*.py).
"""
