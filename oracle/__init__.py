"""FP64 CPU oracle of the grid-overlay FD method -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline
and reference legs) may import this package.  See ``oracle/gofd.py``.
"""
from .gofd import *  # noqa: F401,F403
from . import gofd  # noqa: F401
