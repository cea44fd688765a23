"""GB300-native block Jacobi sweeping preconditioner for the 2-D Helmholtz equation.

The compute path is the CUDA library ``libhelm.so`` (C ABI in include/helm.h),
built in-tree by :mod:`paper_2209_10886_gb300.build`; :mod:`.helm` is its
ctypes binding.
"""
from .helm import (HelmError, MisfitFn, Problem, default_opts, habc_side_operator, header_functions, lib,
                   misfit_grad_sharded, reduce_misfit, schedule_info, source_shard)

__all__ = ["HelmError", "MisfitFn", "Problem", "default_opts", "habc_side_operator", "header_functions", "lib",
           "misfit_grad_sharded", "reduce_misfit", "schedule_info", "source_shard"]
