"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark.  This package holds no arithmetic of the KPM method."""
from . import rng, hamiltonians, vectors, workloads  # noqa: F401
