"""GB300 (sm_103a) library for symmetry-adapted matrix-free H.x and Lanczos.

The compute path is libed.so (hand-written CUDA, C ABI in include/ed.h);
`ed` is its thin ctypes binding.
"""
from .ed import (ED_C64, ED_C128, ED_F32, ED_F64, Basis, BasisSUN, Batch, EdError, Hamiltonian, lib,  # noqa: F401
                 band_eigs, report_dict, representatives, sector_tables, tridiag_eigs)
