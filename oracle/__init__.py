"""Independent FP64 CPU oracle for the grid-integration path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the CUDA library.
"""
from .oracle import Oracle, build_oracle  # noqa: F401
