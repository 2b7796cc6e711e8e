"""FP64 CPU oracle for the FCG-NO hot path (test infrastructure only).

This package is the slow, plain reference that the CUDA library is checked against.
Only the test-suite, the smoke check in ``__graft_entry__`` and the CPU-baseline leg of
``bench.py`` may import it; the library itself never does, and this package never imports
the library. It shares no code, table or constant generator with the CUDA path.
"""
from .fcgno_oracle import *  # noqa: F401,F403
