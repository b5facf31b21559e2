"""Seeded start vectors for the stochastic trace.

Random-phase vectors have unit-modulus entries exp(2*pi*i*u) with u drawn
from SplitMix64 stream 1 at index r*N + i, so column r does not depend on
the block width R.  The library and the oracle each draw the same vectors
from a seed on their own; this module builds them explicitly for the entry
points that take a caller-supplied start block, and builds basis vectors
for exact traces.
"""
import numpy as np

from . import rng


def random_phase_block(seed, n, cols):
    """complex128[n, len(cols)] (row-major), column k = random-phase vector cols[k]."""
    cols = np.atleast_1d(np.asarray(cols, dtype=np.int64))
    idx = (cols[None, :] * n + np.arange(n, dtype=np.int64)[:, None]).astype(np.uint64)
    u = rng.uniform(seed, rng.STREAM_PHASES, idx)
    return np.exp(2j * np.pi * u)


def basis_block(n, first, count):
    """complex128[n, count] whose column k is the unit vector e_{first+k}."""
    v = np.zeros((n, count), dtype=np.complex128)
    v[np.arange(first, first + count), np.arange(count)] = 1.0
    return v


def rows_block(n, rows):
    """complex128[n, len(rows)] whose column k is the unit vector e_{rows[k]}."""
    rows = np.atleast_1d(np.asarray(rows, dtype=np.int64))
    v = np.zeros((n, rows.size), dtype=np.complex128)
    v[rows, np.arange(rows.size)] = 1.0
    return v


def plane_wave_block(dims, norb, q, orb):
    """complex128[n, R] of Bloch waves on a lattice of dims = (nx, ny, nz)
    sites with norb orbitals per site, row i = norb*(x + nx*(y + ny*z)) + a:
    column r is exp(2 pi i q_r . (x, y, z)) / sqrt(sites) on orbital orb[r]
    of every site and zero on the other orbitals."""
    nx, ny, nz = dims
    q = np.asarray(q, dtype=np.float64).reshape(-1, 3)
    orb = np.atleast_1d(np.asarray(orb, dtype=np.int64))
    sites = nx * ny * nz
    s = np.arange(sites)
    x, y, z = s % nx, (s // nx) % ny, s // (nx * ny)
    v = np.zeros((sites * norb, q.shape[0]), dtype=np.complex128)
    for r in range(q.shape[0]):
        phase = q[r, 0] * x + q[r, 1] * y + q[r, 2] * z
        v[norb * s + orb[r], r] = np.exp(2j * np.pi * phase) / np.sqrt(sites)
    return v
