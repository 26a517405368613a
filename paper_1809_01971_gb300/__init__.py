"""GB300 (sm_103a) library for the low-rank PCG solve of the fractional optimal-control
equation (beta^2 A^-alpha + gamma A^alpha) u = beta y_Omega (Heidel, Khoromskaia,
Khoromskij, Schulz, arXiv:1809.01971).

The compute path is libfc.so (CUDA kernels behind the C ABI of include/fc.h); this
package holds its build script and the ctypes binding :mod:`.fc`.

Concurrent solves (``fc_solve_batched``, one library worker stream per solve in flight) need
more hardware work queues than CUDA's default of 8: with 8, streams share queues and their
launches serialise behind each other.  Importing the package therefore sets ``CUDA_DEVICE_MAX_CONNECTIONS`` to
32 unless the caller set it.  CUDA reads it when the context is created, so the setting
counts only if the package is imported before the process first touches the GPU.
"""
import os as _os

_os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from .fc import (CP, FCError, Handle, fc_apply, fc_apply_trunc, fc_autotune, fc_autotune_batched, fc_destroy,
                 fc_dgemm, fc_full_solve, fc_get_info, fc_get_schedule, fc_get_symbol, fc_inner, fc_inner_static, fc_last_cuda_error, fc_launch_count, fc_prof_enable,
                 fc_prof_read, fc_precond, fc_set_schedule, fc_set_wait_limit, fc_set_workspace, fc_setup, fc_solve, fc_solve_batched, fc_state,
                 fc_strerror, fc_symeig, fc_to_full, fc_truncate, fc_workspace_size, lib)

__all__ = ["CP", "FCError", "Handle", "fc_apply", "fc_apply_trunc", "fc_autotune", "fc_autotune_batched",
           "fc_destroy", "fc_dgemm", "fc_full_solve", "fc_get_info", "fc_get_schedule", "fc_get_symbol", "fc_inner", "fc_inner_static", "fc_last_cuda_error",
           "fc_launch_count", "fc_prof_enable", "fc_prof_read", "fc_precond", "fc_set_schedule", "fc_set_wait_limit", "fc_set_workspace",
           "fc_setup", "fc_solve", "fc_solve_batched", "fc_state", "fc_strerror", "fc_symeig",
           "fc_to_full", "fc_truncate", "fc_workspace_size", "lib"]
