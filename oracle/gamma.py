"""Oracle: Euclidean gamma matrices (test infrastructure only).

The paper (Sec. 1) fixes only that D carries 4 spin x 3 colour components per
site.  Reading: Hermitian chiral (Weyl) basis,
    g_k = [[0, -i s_k], [i s_k, 0]]  (k = 1, 2, 3 <-> mu = 0, 1, 2),
    g_4 = [[0, 1], [1, 0]]           (mu = 3, time),
with {g_mu, g_nu} = 2 delta_{mu nu} and g5 = g1 g2 g3 g4 = diag(1, 1, -1, -1),
so gamma5's +1 chirality is spins {0, 1} and -1 is spins {2, 3}.
"""
import numpy as np

_s1 = np.array([[0, 1], [1, 0]], np.complex128)
_s2 = np.array([[0, -1j], [1j, 0]], np.complex128)
_s3 = np.array([[1, 0], [0, -1]], np.complex128)
_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), np.complex128)


def _blk(a, b, c, d):
    return np.block([[a, b], [c, d]])


GAMMA = np.array([_blk(_Z2, -1j * s, 1j * s, _Z2) for s in (_s1, _s2, _s3)]
                 + [_blk(_Z2, _I2, _I2, _Z2)])
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ID4 = np.eye(4, dtype=np.complex128)
