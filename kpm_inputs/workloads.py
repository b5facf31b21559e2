"""The synthetic workloads: topological-insulator lattices with seeded disorder.

They stand in for the paper's own runs (its application section and the
performance sections use such lattices, e.g. 100x100x40, with R = 32 random
vectors and M = 2000 moments at scale); no dataset is involved.
"""
import numpy as np

from . import rng

# name: lattice, disorder strength gamma, M moments, R vectors, seed
TI_SMALL = dict(name="ti_8x8x8_fp64", dims=(8, 8, 8), gamma=0.5, M=256, R=4, seed=0)
TI_64 = dict(name="ti_64x64x64_fp64", dims=(64, 64, 64), gamma=1.0, M=2000, R=32, seed=1,
             chunk_height=32, sigma=256)
TI_LARGE = dict(name="ti_240x240x120_fp64", dims=(240, 240, 120), gamma=2.0, M=1024, R=32, seed=2,
                tile_y=24)
TI_64_FP32 = dict(name="ti_64x64x64_fp32", dims=(64, 64, 64), gamma=1.0, M=1024, R=32, seed=2)
R_SWEEP = (1, 4, 8, 16, 32, 64)


def ensemble(count=64, seed=3):
    """Problem list of the batched ensemble: lattice sizes Nx, Ny in 16..96,
    Nz in 16..48, gamma uniform in [0, 4], even M uniform in [512, 4096],
    R from {8, 16, 32, 64}.  Each problem p draws from stream 2 at indices
    8p..8p+5 and gets its own disorder seed."""
    probs = []
    for p in range(count):
        u = rng.uniform(seed, 2, np.arange(8 * p, 8 * p + 6, dtype=np.uint64))
        nx = 16 + int(u[0] * 81)
        ny = 16 + int(u[1] * 81)
        nz = 16 + int(u[2] * 33)
        gamma = 4.0 * float(u[3])
        M = 2 * (256 + int(u[4] * 1793))
        R = (8, 16, 32, 64)[int(u[5] * 4)]
        probs.append(dict(dims=(nx, ny, nz), gamma=gamma, M=M, R=R, seed=1000 * seed + p))
    return probs
