"""GB300-native matrix-free high-order h-/p-multigrid (libhmg) and its Python binding.

The numerical work lives in the CUDA library ``libhmg.so`` (sources in ``csrc/``, C ABI in
``include/hmg.h``); ``hmg`` is a ctypes binding that only marshals arguments.
"""
from .hmg import (Desc, HmgError, Problem, host_basis, host_hessenberg_max_real_eig, launch_count, lib,  # noqa: F401
                  make_desc, noalloc_lengths, restrict_noalloc, solve_batched)
from .hmg import BatchPlan, Server, desc_ndof, estimate_bytes, measure_peak  # noqa: F401
