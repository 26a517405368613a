"""GB300 (sm_103a) library for the low-rank PCG solve of the fractional optimal-control
equation (beta^2 A^-alpha + gamma A^alpha) u = beta y_Omega (Heidel, Khoromskaia,
Khoromskij, Schulz, arXiv:1809.01971).

The compute path is libfc.so (CUDA kernels behind the C ABI of include/fc.h); this
package holds its build script and the ctypes binding :mod:`.fc`.
"""
from .fc import (CP, FCError, Handle, fc_apply, fc_apply_trunc, fc_dgemm, fc_full_solve, fc_get_symbol, fc_inner,
                 fc_inner_static, fc_launch_count, fc_prof_enable, fc_prof_read, fc_precond, fc_setup, fc_solve, fc_solve_batched, fc_state, fc_symeig, fc_to_full, fc_truncate, lib)

__all__ = ["CP", "FCError", "Handle", "fc_apply", "fc_apply_trunc", "fc_dgemm", "fc_full_solve", "fc_get_symbol", "fc_inner", "fc_inner_static", "fc_launch_count", "fc_prof_enable", "fc_prof_read",
           "fc_precond", "fc_setup", "fc_solve", "fc_solve_batched", "fc_state", "fc_symeig", "fc_to_full", "fc_truncate", "lib"]
