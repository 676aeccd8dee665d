"""CPU FP64 oracle for the symmetry-adapted H.x path -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline arm may
import this package.  It shares no code with the CUDA library
(paper_2210_03511_gb300); the two meet only through the seeded inputs of
`edinputs`.  Every function is pinned by tests/test_oracle_*.py against
closed forms, the thesis's worked examples, invariants and brute force.
"""
from .core import (apply, basis, binom, build, chirality_sum, correlation_matrix, csr, csr_chunked, dense_sz, evolve,  # noqa: F401
                   lowest_eigs, nematic, num_threads, plain_state, product_expectation, projector_matrix, rep,
                   restrict, rows, sector_dim_formula, set_num_threads, sz_spectrum, sz_states,
                   triangle_expectation, lorentzians)
from .ops import bond_matrix, chirality_matrix  # noqa: F401
from . import sun  # noqa: F401  (SU(N) exchange models in the d-ary encoding)
