"""Counter-based uniform random numbers from the SplitMix64 generator.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) advances a 64-bit state by the odd constant
GOLDEN and returns mix(state).  Because the state after k steps is simply
``state0 + k*GOLDEN``, its k-th output can be computed directly, which makes
it counter-based: any element of any stream is available without generating
the ones before it.

The streams used for the synthetic inputs are defined as

    key(seed, stream)        = mix(seed + (stream + 1) * GOLDEN)
    bits(seed, stream, idx)  = mix(key(seed, stream) + (idx + 1) * GOLDEN)
    u(seed, stream, idx)     = (bits >> 11) * 2**-53        in [0, 1)

Stream 0 draws the on-site disorder of the lattice Hamiltonian (index =
lattice site).  Stream 1 is reserved for the random start vectors of the
stochastic trace (index = r*N + i); those are drawn inside the library and
inside the oracle, each from this same published definition.
"""
import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
MIX_MUL1 = 0xBF58476D1CE4E5B9
MIX_MUL2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

STREAM_DISORDER = 0
STREAM_PHASES = 1


def _mix_array(z):
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX_MUL1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX_MUL2)
    return z ^ (z >> np.uint64(31))


def mix_int(z):
    """SplitMix64 output function on one Python int."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * MIX_MUL1) & MASK64
    z = ((z ^ (z >> 27)) * MIX_MUL2) & MASK64
    return z ^ (z >> 31)


def stream_key(seed, stream):
    return mix_int((seed + (stream + 1) * GOLDEN) & MASK64)


def bits(seed, stream, index):
    """64 random bits for each entry of ``index`` (array of non-negative ints)."""
    key = np.uint64(stream_key(int(seed), int(stream)))
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = key + (idx + np.uint64(1)) * np.uint64(GOLDEN)
    return _mix_array(z)


def uniform(seed, stream, index):
    """Uniform doubles in [0, 1) with 53 random bits each."""
    b = bits(seed, stream, index)
    return (b >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
