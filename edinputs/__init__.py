"""Seeded synthetic inputs shared by the CUDA library's tests and the CPU oracle.

Holds the problem statement only (clusters, symmetry permutations, characters,
site ordering) and counter-based random vectors; none of the method's
arithmetic lives here.
"""
from . import configs, lattice, vectors  # noqa: F401
