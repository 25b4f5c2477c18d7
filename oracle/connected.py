"""Oracle: the connected pseudoscalar two-point function and its two-level
multigrid decomposition (Sec. 4, Eqs. 16-20 with L = 2) -- test
infrastructure only.

  G(t) = (1/T) sum_t' tr[ D^{-1}(t+t', t') g5 D^{-1}(t', t+t') g5 ]     (Eq. 16)

(trace over space, spin and colour; time indices modulo T).  Level
operators (Eqs. 17-18) with two levels, read as fine-space operators whose
(t+t', t') blocks are taken on fine timeslices:

  B_1 = D^{-1} - P D_c^{-1} P^dag,      B_2 = P D_c^{-1} P^dag,

so that B_1 + B_2 = D^{-1} (Eq. 10) and, the definition being bilinear,

  G(t) = sum_{i,j} G_ij(t),
  G_ij(t) = (1/T) sum_t' tr[ B_i(t+t', t') g5 B_j(t', t+t') g5 ]         (Eqs. 19-20).

Stochastic estimate (the standard estimator of a connected pseudoscalar
correlator): D^{-1} and P D_c^{-1} P^dag are gamma5-hermitian (P keeps the
chirality halves apart), so B_j(t', t+t') = g5 B_j(t+t', t')^dag g5 and
G_ij(t) = (1/T) sum_t' tr[ B_i(t+t', t') B_j(t+t', t')^dag ].  With Rademacher
noise eta supported on timeslice t' and y_k = B_k eta,

  sample_ij(t) = (1/T) sum_t' sum_{x in t+t'} y_j(x)^dag y_i(x),

whose expectation is G_ij(t) since E[eta eta^dag] = 1 on timeslice t'.
"""
import numpy as np

from .noise import rademacher
from .wilson import gamma5_full, timeslice_of_dof


def _g5(n):
    return gamma5_full(n // 12)


def correlator_exact(A, B, dims):
    """(1/T) sum_t' tr[A(t+t', t') g5 B(t', t+t') g5] for dense fine-space
    operators A, B (the definition of Eqs. 16 and 20), complex array (T,)."""
    T = dims[3]
    n = A.shape[0]
    ts = timeslice_of_dof(dims)
    g5 = _g5(n)
    out = np.zeros(T, np.complex128)
    for t in range(T):
        for tp in range(T):
            a = np.where(ts == (t + tp) % T)[0]
            b = np.where(ts == tp)[0]
            Ab = A[np.ix_(a, b)]                              # A(t+t', t')
            M = g5[b][:, None] * B[np.ix_(b, a)] * g5[a][None, :]   # g5 B(t', t+t') g5
            out[t] += np.trace(Ab @ M) / T
    return out


def level_operators(Dinv, Pd, Dcinv):
    """B_1 = D^{-1} - P D_c^{-1} P^dag and B_2 = P D_c^{-1} P^dag (dense)."""
    B2 = Pd @ Dcinv @ Pd.conj().T
    return Dinv - B2, B2


# noise samples of the separately sampled (2,2) term: i | LEVEL2_STREAM
LEVEL2_STREAM = 1 << 21


def samples(solve, solve_coarse, P, dims, seed, N1, N2):
    """Per-sample estimates of G_ij(t) from time-diluted Rademacher noise:
    returns (S1 (N1, 4, T) for (i, j) = (1,1), (1,2), (2,1), (2,2) from noise
    samples 0 .. N1-1, and S2 (N2, T) for (2, 2) from the independent noise
    samples i | LEVEL2_STREAM).  Each sample puts the noise on every source
    timeslice t' in turn.  The (2, 2) term needs only coarse solves, so the
    estimate samples it on its own (N2 samples, typically more than N1): G is
    mean(S11 + S12 + S21) + mean(S22), with variance
    var(S11 + S12 + S21) / N1 + var(S22) / N2.  S1's (2, 2) column (same noise
    as level 1) gives the plain estimator |y_1 + y_2|^2 for comparison."""
    X, Y, Z, T = dims
    n = 12 * X * Y * Z * T
    ts = timeslice_of_dof(dims)
    S1 = np.zeros((N1, 4, T), np.complex128)
    S2 = np.zeros((N2, T), np.complex128)
    for level, N in ((1, N1), (2, N2)):
        for i in range(N):
            eta = rademacher(seed, i if level == 1 else i | LEVEL2_STREAM, n)
            for tp in range(T):
                v = np.where(ts == tp, eta, 0).astype(np.complex128)
                y2 = P @ solve_coarse(P.conj().T @ v)
                y1 = solve(v) - y2 if level == 1 else None
                for t in range(T):
                    m = ts == (t + tp) % T
                    if level == 2:
                        S2[i, t] += np.vdot(y2[m], y2[m]) / T
                    else:
                        S1[i, 0, t] += np.vdot(y1[m], y1[m]) / T
                        S1[i, 1, t] += np.vdot(y2[m], y1[m]) / T   # (1,2): y_2^dag y_1
                        S1[i, 2, t] += np.vdot(y1[m], y2[m]) / T   # (2,1): y_1^dag y_2
                        S1[i, 3, t] += np.vdot(y2[m], y2[m]) / T
    return S1, S2


def estimate(S1, S2):
    """(G (6, T): means of (1,1), (1,2), (2,1), (2,2) [from S2], of the total,
    and of the plain estimator S11 + S12 + S21 + S22 on the level-1 noise;
    var (6, T): variances of those means)."""
    lvl1 = S1[:, :3].sum(1)
    G = np.stack([S1[:, 0].mean(0), S1[:, 1].mean(0), S1[:, 2].mean(0), S2.mean(0),
                  lvl1.mean(0) + S2.mean(0), S1.sum(1).mean(0)])
    v = lambda a: np.sum(np.abs(a - a.mean(0)) ** 2, axis=0) / (a.shape[0] - 1) / a.shape[0]
    var = np.stack([v(S1[:, 0]), v(S1[:, 1]), v(S1[:, 2]), v(S2), v(lvl1) + v(S2), v(S1.sum(1))])
    return G, var
