"""Oracle: the D^{-1} eta products of Sec. 1 (test infrastructure only).

Sec. 1: the estimators need only products D^{-1} eta, obtained by solving a
linear system with D as the system matrix.  The paper names no Krylov
method; BiCGStab (van der Vorst 1992) in FP64 on the full, unpreconditioned
operator is used here, and dense LU for exact inverses on tiny lattices.
"""
import numpy as np
import scipy.linalg as sla


def bicgstab(apply_A, b, tol=1e-12, max_iter=20000, x0=None):
    """Textbook BiCGStab for A x = b (complex, FP64).  Stops when the
    recursively updated residual satisfies ||r|| <= tol ||b||, then returns
    (x, iterations, true relative residual)."""
    b = np.asarray(b, np.complex128)
    shape = b.shape
    b = b.reshape(-1)
    A = lambda v: np.asarray(apply_A(v.reshape(shape))).reshape(-1)
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, np.complex128).reshape(-1).copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x.reshape(shape), 0, 0.0
    r = b - A(x)
    rhat = r.copy()
    rho_old = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b); p = np.zeros_like(b)
    it = 0
    while it < max_iter and np.linalg.norm(r) > tol * bnorm:
        rho = np.vdot(rhat, r)
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = A(p)
        alpha = rho / np.vdot(rhat, v)
        s = r - alpha * v
        t = A(s)
        omega = np.vdot(t, s) / np.vdot(t, t)
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        it += 1
    true_res = np.linalg.norm(b - A(x)) / bnorm
    return x.reshape(shape), it, true_res


def dense_inverse(Dmat):
    """D^{-1} of a dense (or scipy sparse) matrix via LU."""
    if hasattr(Dmat, 'toarray'):
        Dmat = Dmat.toarray()
    lu = sla.lu_factor(Dmat)
    return sla.lu_solve(lu, np.eye(Dmat.shape[0], dtype=np.complex128))


def exact_traces(Dinv, dims, gamma5):
    """Exact per-timeslice traces of B D^{-1} from a dense inverse:
    tr[B D^{-1}(t, t)] for t = 0..T-1, B = gamma5 (x) 1 if gamma5 else 1.
    Returns a complex array of length T (its sum is tr(B D^{-1}))."""
    from .wilson import gamma5_full, timeslice_of_dof
    X, Y, Z, T = dims
    V = X * Y * Z * T
    diag = np.diag(Dinv).copy()
    if gamma5:
        diag = diag * gamma5_full(V)
    ts = timeslice_of_dof(dims)
    return np.array([diag[ts == t].sum() for t in range(T)])
