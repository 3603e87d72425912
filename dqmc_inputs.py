"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module holds no arithmetic of the method: only seeded random fields,
matrices and parameter sets shaped like the paper's workloads (Sec. III:
kagome tori L = 4..36, 3 sites per cell, dtau = 0.1, Ising fields s = +-1).
Random numbers that the Markov chain itself draws are not made here: both the
CUDA path and the oracle generate those with Philox4x32-10 from the seed.
"""

import numpy as np

# Workloads. Common: t = 1, mu = -1 (Dirac filling at U = 0), dtau = 0.1,
# attractive |U| = 4 passed with the paper's sign (U < 0 is attraction).
WORKLOADS = {
    "L4_fp64": dict(L=4, beta=2.0, dtau=0.1, U=-4.0, mu=-1.0, seed=1, k=8, n_stab=10,
                    precision="fp64", warmup=200, measure=200),
    "L12_fp64": dict(L=12, beta=12.0, dtau=0.1, U=-4.0, mu=-1.0, seed=1, k=32, n_stab=10,
                     precision="fp64", sweeps=1000),
    "L24_mixed": dict(L=24, beta=24.0, dtau=0.1, U=-4.0, mu=-1.0, seed=1, k=32, n_stab=8,
                      precision="mixed"),
    "L36_mixed": dict(L=36, beta=36.0, dtau=0.1, U=-4.0, mu=-1.0, seed=1, k=32, n_stab=8,
                      precision="mixed"),
}


def random_field(M, N, seed):
    """Uniform +-1 Ising field, shape (M, N), int8, slice-major."""
    rng = np.random.default_rng(seed)
    return np.where(rng.random((M, N)) < 0.5, 1, -1).astype(np.int8)


def random_matrix(rows, cols, seed, scale=1.0):
    """Dense FP64 matrix with i.i.d. normal entries."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((rows, cols))


def random_green_like(N, seed):
    """A matrix with the magnitude structure of an equal-time G: diagonal near
    1/2, off-diagonal entries decaying like a short-range correlation."""
    rng = np.random.default_rng(seed)
    A = 0.05 * rng.standard_normal((N, N))
    A[np.arange(N), np.arange(N)] = 0.5 + 0.2 * rng.standard_normal(N)
    return A


def random_uniforms(n, seed):
    rng = np.random.default_rng(seed)
    return rng.random(n)
