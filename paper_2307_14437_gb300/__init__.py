"""GB300-native grid-overlay FD method (GoFD) for the fractional Laplacian.

The compute path is the CUDA library ``libgofd.so`` (C ABI in ``include/gofd.h``);
this package is its thin binding.  Build it with ``build_native.build()``.
"""
from .gofd import GofdError, Group, Problem, grid_key, group_key, solve_many  # noqa: F401

__all__ = ["Problem", "Group", "GofdError", "grid_key", "group_key", "solve_many"]
