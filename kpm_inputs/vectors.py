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
