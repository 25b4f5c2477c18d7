"""Oracle: stochastic trace estimators of the paper (test infrastructure only).

All estimators target tr[B D^{-1}(t, t)] per timeslice t, with B = 1 or
gamma5 (x) 1 (Sec. 4, Eq. 21, O(t) = tr[Gamma5(t) D^{-1}(t, t)]), and return
the per-sample values X_i(t) so that the mean and the sample variance can be
formed.  A per-sample value is the quadratic form of the paper restricted to
the dofs of timeslice t:  X(t) = sum_{j in t} conj(v_j) (B D^{-1} v)_j.

  hutchinson   Eq. 3 with Rademacher vectors (Sec. 1); optional time dilution
               (v restricted to one timeslice per solve).
  probing      Eq. 14 with the probing vectors of Eq. 13 (Rademacher entries on
               one colour of the torus colouring, Eq. 15), times spin-colour
               dilution (Sec. 3: 12 components for full dilution).  The
               printed Eq. 14 lacks the dagger on the left vector; it is read
               as v^dagger (equal to v^T for real v).
  mlmc2        the two-level multigrid MLMC estimator (Eqs. 9-12 with L = 2):
               X_1 = eta^dag B (D^{-1} - P D_c^{-1} P^dag) eta  on fine noise,
               X_2 = (P xi)^dag B (P D_c^{-1} xi)             on coarse noise,
               the second being tr(B P D_c^{-1} P^dag) = tr(P^dag B P D_c^{-1}).
  mlmc2_probe  the combination the paper proposes in its outlook (Sec. 6):
               the level-1 term tr(B M_1) of Eq. 12 estimated with the probing
               x dilution vectors of Eqs. 13-14 (optionally one timeslice per
               vector) instead of plain Rademacher vectors; level 2 as mlmc2.
  mlmc3        the three-level estimator (Eqs. 9-12 with L = 3):
               X_1 = eta^dag B (D^{-1} - P_1 D_2^{-1} P_1^dag) eta          fine noise,
               X_2 = (P_1 xi)^dag B P_1 (D_2^{-1} - P_2 D_3^{-1} P_2^dag) xi  level-2 noise,
               X_3 = (P_1 P_2 zeta)^dag B (P_1 P_2 D_3^{-1} zeta)           level-3 noise.
  mlmc_allocation  Eq. 6: the number of samples per level that minimises the
               total cost sum_l N_l C_l for a target variance eps^2.

`solve(v)` is any callable returning D^{-1} v for a flat length-12V vector.
"""
import numpy as np

from .noise import rademacher, COARSE_STREAM
from .wilson import gamma5_full, timeslice_of_dof


def contract(v, y, dims, gamma5):
    """X(t) = sum_{j in timeslice t} conj(v_j) (B y)_j, complex array (T,)."""
    X, Y, Z, T = dims
    V = X * Y * Z * T
    by = y * gamma5_full(V) if gamma5 else y
    prod = np.conj(v) * by
    return prod.reshape(T, -1).sum(axis=1)


def hutchinson(solve, dims, seed, N, gamma5, time_dilution=False, sample0=0):
    """Per-sample X_i(t), shape (N, T)."""
    X, Y, Z, T = dims
    n = 12 * X * Y * Z * T
    ts = timeslice_of_dof(dims)
    out = np.zeros((N, T), np.complex128)
    for i in range(N):
        eta = rademacher(seed, sample0 + i, n).astype(np.complex128)
        if time_dilution:
            for t in range(T):
                v = np.where(ts == t, eta, 0)
                out[i] += contract(v, solve(v), dims, gamma5)
        else:
            out[i] = contract(eta, solve(eta), dims, gamma5)
    return out


def probing_masks(col, nc, dilution):
    """Boolean masks (nc*dilution, 12V) of the probing x dilution vectors:
    colour c of the site (col: per-site colours) and, for dilution 12, the
    spin-colour component k = 3*spin + colour of the dof."""
    V = col.shape[0]
    site_col = np.repeat(col, 12)
    comp = np.tile(np.arange(12), V)
    masks = []
    for c in range(nc):
        for k in range(dilution):
            m = site_col == c
            if dilution == 12:
                m = m & (comp == k)
            masks.append(m)
    return np.array(masks)


def probing(solve, dims, seed, N, gamma5, col, nc, dilution, sample0=0):
    """Per-sample X_i(t) = sum over colours and dilution components, (N, T)."""
    X, Y, Z, T = dims
    n = 12 * X * Y * Z * T
    masks = probing_masks(col, nc, dilution)
    out = np.zeros((N, T), np.complex128)
    for i in range(N):
        eta = rademacher(seed, sample0 + i, n).astype(np.complex128)
        for m in masks:
            v = np.where(m, eta, 0)
            out[i] += contract(v, solve(v), dims, gamma5)
    return out


def mlmc2(solve, solve_coarse, P, dims, seed, N1, N2, gamma5, sample0=0):
    """Per-sample level values (X1 (N1, T), X2 (N2, T)) of the 2-level estimator."""
    X, Y, Z, T = dims
    n = 12 * X * Y * Z * T
    ncd = P.shape[1]
    X1 = np.zeros((N1, T), np.complex128)
    for i in range(N1):
        eta = rademacher(seed, sample0 + i, n).astype(np.complex128)
        z = solve(eta)
        w = P @ solve_coarse(P.conj().T @ eta)
        X1[i] = contract(eta, z - w, dims, gamma5)
    X2 = np.zeros((N2, T), np.complex128)
    for i in range(N2):
        xi = rademacher(seed, (sample0 + i) | COARSE_STREAM, ncd).astype(np.complex128)
        X2[i] = contract(P @ xi, P @ solve_coarse(xi), dims, gamma5)
    return X1, X2


def mlmc2_probe(solve, solve_coarse, P, dims, seed, N1, N2, gamma5, col, nc, dilution, time_dilution=False,
                sample0=0, coarse_col=None, coarse_nc=1, coarse_dil=1):
    """Per-sample level values (X1 (N1, T), X2 (N2, T)) of the two-level
    estimator with probing on level 1 (Sec. 6 outlook; Eqs. 12-14): for sample
    i, X1_i = sum over the probing x dilution (x timeslice) vectors v of eta_i
    of v^dag B (D^{-1} v - P D_c^{-1} P^dag v).  Level 2 as in mlmc2, or, with
    coarse_col (per-coarse-site colours of a colouring of the coarse torus),
    probed as well: X2_i = sum over the coarse probing vectors xi (coarse
    noise sample i masked to one colour and, for coarse_dil = 2 nv, one
    coarse dof of the site) of (P xi)^dag B (P D_c^{-1} xi)."""
    X, Y, Z, T = dims
    n = 12 * X * Y * Z * T
    masks = probing_masks(col, nc, dilution)
    if time_dilution:
        ts = timeslice_of_dof(dims)
        masks = [m & (ts == t) for m in masks for t in range(T)]
    X1 = np.zeros((N1, T), np.complex128)
    for i in range(N1):
        eta = rademacher(seed, sample0 + i, n)
        for m in masks:
            v = np.where(m, eta, 0).astype(np.complex128)
            X1[i] += contract(v, solve(v) - P @ solve_coarse(P.conj().T @ v), dims, gamma5)
    if coarse_col is None:
        _, X2 = mlmc2(solve, solve_coarse, P, dims, seed, 0, N2, gamma5, sample0)
        return X1, X2
    ncd = P.shape[1]
    m = ncd // len(coarse_col)                   # coarse dofs per coarse site
    site_col = np.repeat(np.asarray(coarse_col), m)
    comp = np.tile(np.arange(m), len(coarse_col))
    X2 = np.zeros((N2, T), np.complex128)
    for i in range(N2):
        xi = rademacher(seed, (sample0 + i) | COARSE_STREAM, ncd)
        for c in range(coarse_nc):
            for k in range(coarse_dil):
                msk = (site_col == c) & ((comp == k) if coarse_dil > 1 else True)
                v = np.where(msk, xi, 0).astype(np.complex128)
                X2[i] += contract(P @ v, P @ solve_coarse(v), dims, gamma5)
    return X1, X2


LEVEL3_STREAM = 1 << 24


def mlmc3(solve, solve2, solve3, P1, P2, dims, seed, N1, N2, N3, gamma5):
    """Per-sample level values (X1 (N1, T), X2 (N2, T), X3 (N3, T)) of the
    three-level estimator (Eq. 12 with L = 3).  Level-2 noise: coarse noise
    samples i | COARSE_STREAM; level-3 noise: samples i | LEVEL3_STREAM."""
    X, Y, Z, T = dims
    n = 12 * X * Y * Z * T
    n2, n3 = P1.shape[1], P2.shape[1]
    X1 = np.zeros((N1, T), np.complex128)
    for i in range(N1):
        eta = rademacher(seed, i, n).astype(np.complex128)
        X1[i] = contract(eta, solve(eta) - P1 @ solve2(P1.conj().T @ eta), dims, gamma5)
    X2 = np.zeros((N2, T), np.complex128)
    for i in range(N2):
        xi = rademacher(seed, i | COARSE_STREAM, n2).astype(np.complex128)
        a = solve2(xi) - P2 @ solve3(P2.conj().T @ xi)
        X2[i] = contract(P1 @ xi, P1 @ a, dims, gamma5)
    X3 = np.zeros((N3, T), np.complex128)
    for i in range(N3):
        zeta = rademacher(seed, i | LEVEL3_STREAM, n3).astype(np.complex128)
        X3[i] = contract(P1 @ (P2 @ zeta), P1 @ (P2 @ solve3(zeta)), dims, gamma5)
    return X1, X2, X3


def mlmc_allocation(V, C, eps):
    """Eq. 6: N_l = eps^-2 sqrt(V_l / C_l) sum_i sqrt(V_i C_i), the minimiser
    of sum_l N_l C_l subject to sum_l V_l / N_l = eps^2 (real N_l).  Returns
    (continuous N_l, integer N_l = ceil, at least 1)."""
    V = np.asarray(V, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    s = np.sum(np.sqrt(V * C))
    Nc = np.sqrt(V / C) * s / eps ** 2
    return Nc, np.maximum(np.ceil(Nc - 1e-9 * Nc), 1).astype(np.int64)


def mean_and_variance(samples):
    """Mean over samples and the sample variance s^2 = sum |X_i - mean|^2/(N-1)
    (complex modulus), for each column and for the total over columns.
    Returns (mean (T,), var (T,), mean_total, var_total)."""
    s = np.asarray(samples)
    N = s.shape[0]
    tot = s.sum(axis=1)
    mean = s.mean(axis=0)
    mt = tot.mean()
    if N < 2:
        return mean, np.full(s.shape[1], np.nan), mt, np.nan
    var = (np.abs(s - mean) ** 2).sum(axis=0) / (N - 1)
    vt = (np.abs(tot - mt) ** 2).sum() / (N - 1)
    return mean, var, mt, vt


def hutchinson_variance(A):
    """Eq. 4: V[eta^T A eta] = 1/2 || offdiag(A + A^T) ||_F^2 (Rademacher eta)."""
    S = A + A.T
    S = S - np.diag(np.diag(S))
    return 0.5 * np.sum(np.abs(S) ** 2)


def probing_variance(A, groups):
    """Variance of sum_g v_g^T A v_g when v_g is eta restricted to the dofs of
    group g (colour x dilution component): only pairs i != j in the same group
    contribute, V = 1/2 sum_{i != j, g_i = g_j} |A_ij + A_ji|^2."""
    S = A + A.T
    same = groups[:, None] == groups[None, :]
    np.fill_diagonal(same, False)
    return 0.5 * np.sum(np.abs(S[same]) ** 2)
