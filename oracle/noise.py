"""Oracle: Rademacher noise from a counter-based hash (test infrastructure only).

Sec. 1 asks for vectors with E[eta_j] = 0 and E[conj(eta_j) eta_k] = delta_jk
(Eq. 1) and takes them Rademacher: each entry +1 or -1 with probability 1/2.
The paper fixes no generator.  Reading: every entry is a pure function of
(seed, sample, dof index j), so the oracle and the CUDA path draw identical
vectors without sharing code or state:

    key  = seed XOR (sample << 40) XOR j                    (64-bit)
    h    = splitmix64(key)   -- Steele, Lea & Flood (2014), the output function
           of Vigna's splitmix64: z = key + 0x9E3779B97F4A7C15;
           z = (z ^ z>>30) * 0xBF58476D1CE4E5B9; z = (z ^ z>>27) * 0x94D049BB133111EB;
           h = z ^ z>>31
    eta_j = +1 if the top bit of h is 0, else -1.

Fine-lattice dofs use j = 12*site + 3*spin + colour; coarse-grid noise (the
second MLMC level) uses the same hash with `sample | 2**23`.
"""
import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
COARSE_STREAM = 1 << 23


def splitmix64(key):
    """Vectorised splitmix64 output function on a uint64 array (wraps mod 2^64)."""
    z = np.asarray(key, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def rademacher(seed, sample, n):
    """Real +/-1 vector of length n for noise sample `sample`."""
    with np.errstate(over='ignore'):
        j = np.arange(n, dtype=np.uint64)
        key = np.uint64(seed) ^ (np.uint64(sample) << np.uint64(40)) ^ j
        h = splitmix64(key)
    return 1.0 - 2.0 * (h >> np.uint64(63)).astype(np.float64)
